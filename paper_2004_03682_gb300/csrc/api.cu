// The C ABI of libexpgb (include/exp.h): validation, context lifetime, error
// mapping, the iteration loop with CUDA-graph replay, amplitude I/O.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <string>
#include <cstring>
#include <cstdlib>

#include "ccsd.h"
#include "fs.h"
#include "emu.h"
#include "packed.h"

static thread_local std::string g_err;

#define API_BEGIN try {
#define API_END(ctxp)                                                                  \
  }                                                                                    \
  catch (const ExpError& e) {                                                          \
    g_err = e.msg;                                                                     \
    if (ctxp) (ctxp)->c.err = e.msg;                                                   \
    return e.s;                                                                        \
  }                                                                                    \
  catch (const CudaError& e) {                                                         \
    g_err = std::string(e.where) + ": " + cudaGetErrorString(e.e);                     \
    if (ctxp) (ctxp)->c.err = g_err;                                                   \
    return EXP_ECUDA;                                                                  \
  }                                                                                    \
  catch (const std::exception& e) {                                                    \
    g_err = e.what();                                                                  \
    if (ctxp) (ctxp)->c.err = g_err;                                                   \
    return EXP_EINVAL;                                                                 \
  }

static void check_config(const exp_config* cfg) {
  if (!cfg) throw ExpError{EXP_EINVAL, "null config"};
  if (cfg->n_inst < 1 || cfg->n_occ < 1 || cfg->n_virt < 1) throw ExpError{EXP_EINVAL, "sizes must be >= 1"};
  if (cfg->n_irrep < 1 || cfg->n_irrep > EXP_MAX_G) throw ExpError{EXP_EINVAL, "n_irrep must be in 1..16"};
  if (!cfg->irrep_occ || !cfg->irrep_virt || !cfg->eps_occ || !cfg->eps_virt)
    throw ExpError{EXP_EINVAL, "null irrep or energy array"};
  int so = 0, sv = 0;
  for (int g = 0; g < cfg->n_irrep; ++g) {
    if (cfg->irrep_occ[g] < 0 || cfg->irrep_virt[g] < 0) throw ExpError{EXP_EINVAL, "negative irrep count"};
    so += cfg->irrep_occ[g];
    sv += cfg->irrep_virt[g];
  }
  if (so != cfg->n_occ || sv != cfg->n_virt) throw ExpError{EXP_EINVAL, "irrep counts do not sum to n_occ/n_virt"};
  if (cfg->precision != EXP_FP64 && cfg->precision != EXP_EMU_BF16) throw ExpError{EXP_EINVAL, "bad precision"};
  if (cfg->precision == EXP_EMU_BF16 && (cfg->n_slices < 3 || cfg->n_slices > 6))
    throw ExpError{EXP_EINVAL, "n_slices must be in 3..6"};
  if (cfg->precision == EXP_EMU_BF16 && cfg->n_slices_major != 0 &&
      (cfg->n_slices_major < 3 || cfg->n_slices_major > 6))
    throw ExpError{EXP_EINVAL, "n_slices_major must be 0 or in 3..6"};
  if (cfg->real_arith != 0 && cfg->real_arith != 1) throw ExpError{EXP_EINVAL, "real_arith must be 0 or 1"};
  if (!(cfg->denom_shift >= 0) || !std::isfinite(cfg->denom_shift)) throw ExpError{EXP_EINVAL, "denom_shift must be >= 0"};
  if (cfg->denom_shift > 0 && (cfg->denom_shift_n < 1 || cfg->denom_shift_n > 16))
    throw ExpError{EXP_EINVAL, "denom_shift_n must be in 1..16"};
  if (cfg->diis_dim < 0 || cfg->diis_dim > EXP_MAX_DIIS) throw ExpError{EXP_EINVAL, "diis_dim must be in 0..8"};
  if (!(cfg->conv_tol > 0)) throw ExpError{EXP_EINVAL, "conv_tol must be > 0"};
  if (!(cfg->level_shift >= 0) || !std::isfinite(cfg->level_shift)) throw ExpError{EXP_EINVAL, "level_shift must be >= 0"};
  if (cfg->packed != 0 && cfg->packed != 1) throw ExpError{EXP_EINVAL, "packed must be 0 or 1"};
  if (cfg->n_active < 0 || cfg->n_active > cfg->n_virt) throw ExpError{EXP_EINVAL, "n_active out of range"};
  if (cfg->n_active > 0) {
    if (!cfg->active_virt) throw ExpError{EXP_EINVAL, "null active_virt"};
    std::vector<char> seen(cfg->n_virt, 0);
    for (int k = 0; k < cfg->n_active; ++k) {
      const int a = cfg->active_virt[k];
      if (a < 0 || a >= cfg->n_virt || seen[a]) throw ExpError{EXP_EINVAL, "active_virt: bad or repeated index"};
      seen[a] = 1;
    }
  }
  if (cfg->max_iter < 1) throw ExpError{EXP_EINVAL, "max_iter must be >= 1"};
  for (int64_t k = 0; k < int64_t(cfg->n_inst) * cfg->n_occ; ++k)
    if (!std::isfinite(cfg->eps_occ[k])) throw ExpError{EXP_EINVAL, "non-finite eps_occ"};
  for (int64_t k = 0; k < int64_t(cfg->n_inst) * cfg->n_virt; ++k)
    if (!std::isfinite(cfg->eps_virt[k])) throw ExpError{EXP_EINVAL, "non-finite eps_virt"};
}

extern "C" exp_status exp_create(const exp_config* cfg, const exp_allocator* alloc, void* stream, exp_ctx** out) {
  exp_ctx* x = nullptr;
  API_BEGIN
  if (!out) throw ExpError{EXP_EINVAL, "null out"};
  *out = nullptr;
  check_config(cfg);
  if (!alloc || !alloc->alloc || !alloc->free) throw ExpError{EXP_EINVAL, "null allocator"};
  x = new exp_ctx();
  Ctx& c = x->c;
  c.cfg = *cfg;
  c.cfg.irrep_occ = c.cfg.irrep_virt = nullptr;
  c.cfg.eps_occ = c.cfg.eps_virt = nullptr;
  c.cfg.active_virt = nullptr;
  c.alloc = *alloc;
  c.stream = (cudaStream_t)stream;
  c.G = cfg->n_irrep;
  c.no = cfg->n_occ;
  c.nv = cfg->n_virt;
  c.ninst = cfg->n_inst;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev));
  // Spaces.  With active spinors, every active virtual x gets a ghost occupied
  // spinor g_x (same irrep, orbital energy 0, no integrals); the (0h,1p) sector's
  // electron-attached vectors are carried as the ghosts' amplitudes.  Inside each
  // occupied irrep the real spinors come first, then the ghosts.
  c.no_real = cfg->n_occ;
  c.nact = cfg->n_active;
  c.act.assign(cfg->active_virt, cfg->active_virt + c.nact);
  std::vector<int> virt_irrep(c.nv);
  {
    int a = 0;
    for (int g = 0; g < c.G; ++g)
      for (int k = 0; k < cfg->irrep_virt[g]; ++k) virt_irrep[a++] = g;
  }
  std::vector<int> ghosts_in(c.G, 0);
  for (int k = 0; k < c.nact; ++k) ghosts_in[virt_irrep[c.act[k]]]++;
  c.no = c.no_real + c.nact;
  c.spaces.resize(SP_COUNT);
  for (int s2 = 0; s2 < SP_COUNT; ++s2) {
    Space& sp = c.spaces[s2];
    sp.cnt.resize(c.G);
    for (int g = 0; g < c.G; ++g)
      sp.cnt[g] = s2 == SP_OCC ? cfg->irrep_occ[g] + ghosts_in[g] : cfg->irrep_virt[g];
    sp.off.resize(c.G);
    int o = 0;
    for (int g = 0; g < c.G; ++g) { sp.off[g] = o; o += sp.cnt[g]; }
    sp.n = o;
    sp.gbase = s2 == SP_OCC ? 0 : c.no;
  }
  c.occ_real.assign(c.no, -1);
  c.occ_ghost.assign(c.no, -1);
  {
    int real = 0;
    for (int g = 0; g < c.G; ++g) {
      int l = c.spaces[SP_OCC].off[g];
      for (int k = 0; k < cfg->irrep_occ[g]; ++k) c.occ_real[l++] = real++;
      for (int k = 0; k < c.nact; ++k)
        if (virt_irrep[c.act[k]] == g) c.occ_ghost[l++] = k;
    }
  }
  const int n = c.no + c.nv;
  c.n_gen = c.no_real + c.nv;
  std::vector<double> eps(size_t(c.ninst) * n), eps_fs(size_t(c.ninst) * n);
  for (int k = 0; k < c.ninst; ++k) {
    for (int l = 0; l < c.no; ++l) {
      const int r = c.occ_real[l];
      eps[size_t(k) * n + l] = r >= 0 ? cfg->eps_occ[size_t(k) * c.no_real + r] : 0.0;
      eps_fs[size_t(k) * n + l] =
          r >= 0 ? cfg->eps_occ[size_t(k) * c.no_real + r] : cfg->eps_virt[size_t(k) * c.nv + c.act[c.occ_ghost[l]]];
    }
    for (int a = 0; a < c.nv; ++a) eps[size_t(k) * n + c.no + a] = eps_fs[size_t(k) * n + c.no + a] =
        cfg->eps_virt[size_t(k) * c.nv + a];
  }
  c.d_eps = (double*)c.dalloc(eps.size() * sizeof(double));
  upload(c, c.d_eps, eps.data(), eps.size() * sizeof(double));
  c.d_occreal = (int*)c.dalloc(sizeof(int) * c.no);
  upload(c, c.d_occreal, c.occ_real.data(), sizeof(int) * c.no);
  if (c.nact) {
    c.d_eps_fs = (double*)c.dalloc(eps_fs.size() * sizeof(double));
    upload(c, c.d_eps_fs, eps_fs.data(), eps_fs.size() * sizeof(double));
    std::vector<int> gm(n);
    for (int l = 0; l < c.no; ++l) gm[l] = c.occ_real[l];
    for (int a = 0; a < c.nv; ++a) gm[c.no + a] = c.no_real + a;
    c.d_genmap = (int*)c.dalloc(sizeof(int) * n);
    upload(c, c.d_genmap, gm.data(), sizeof(int) * n);
  }
  c.d_seed = (uint64_t*)c.dalloc(sizeof(uint64_t) * c.ninst);
  c.d_scale = (double*)c.dalloc(sizeof(double) * c.ninst);
  CK(cudaEventCreate(&c.ev0));
  CK(cudaEventCreate(&c.ev1));
  CK(cudaEventCreate(&c.pev0));
  CK(cudaEventCreate(&c.pev1));
  {
    const char* pe = getenv("EXP_PROFILE");
    c.profile = pe && pe[0] == '1';
    // EXP_AUTOTUNE=0: keep the default work decomposition of the emulated products,
    // or the one forced by EXP_KSPLIT_MULT (K-split multiplier) / EXP_GROUP_ROWS
    const char* at = getenv("EXP_AUTOTUNE");
    if (at && at[0] == '0') {
      c.autotune = false;
      if (const char* km = getenv("EXP_KSPLIT_MULT")) c.force_ksplit_mult = std::max(0.0, atof(km));
      if (const char* gr = getenv("EXP_GROUP_ROWS")) c.force_group_rows = std::max(1, atoi(gr));
    }
  }
  ccsd_setup(c);
  CK(cudaStreamSynchronize(c.stream));
  *out = x;
  return EXP_OK;
  }
  catch (const ExpError& e) {
    g_err = e.msg;
    if (x) { x->c.dfree_all(); delete x; }
    return e.s;
  }
  catch (const CudaError& e) {
    g_err = std::string(e.where) + ": " + cudaGetErrorString(e.e);
    if (x) { x->c.dfree_all(); delete x; }
    return EXP_ECUDA;
  }
}

extern "C" void exp_destroy(exp_ctx* x) {
  if (!x) return;
  Ctx& c = x->c;
  cudaStreamSynchronize(c.stream);
  if (c.graph) cudaGraphExecDestroy(c.graph);
  if (c.ev0) cudaEventDestroy(c.ev0);
  if (c.ev1) cudaEventDestroy(c.ev1);
  if (c.pev0) cudaEventDestroy(c.pev0);
  if (c.pev1) cudaEventDestroy(c.pev1);
  if (c.h_stats) cudaFreeHost(c.h_stats);
  staging_release(c);
  fs_release(c);
  try { emu_release(c); } catch (...) {}
  packed_release(c);
  ccsd_release(c);
  c.dfree_all();
  delete x;
}

extern "C" exp_status exp_init_integrals(exp_ctx* x, const uint64_t* seeds, const double* scale_mult,
                                         double* scale_out) {
  API_BEGIN
  if (!x || !seeds) throw ExpError{EXP_EINVAL, "null argument"};
  Ctx& c = x->c;
  if (c.have_integrals) throw ExpError{EXP_ESTATE, "integrals already initialised"};
  upload(c, c.d_seed, seeds, sizeof(uint64_t) * c.ninst);
  std::vector<double> mult(c.ninst, 1.0);
  if (scale_mult)
    for (int k = 0; k < c.ninst; ++k) {
      if (!(scale_mult[k] > 0) || !std::isfinite(scale_mult[k])) throw ExpError{EXP_EINVAL, "scale_mult must be > 0"};
      mult[k] = scale_mult[k];
    }
  ccsd_init_integrals(c, mult.data());
  if (scale_out)
    for (int k = 0; k < c.ninst; ++k) scale_out[k] = c.h_scale[k];
  return EXP_OK;
  API_END(x)
}

static int64_t count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  CK(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CK(cudaGraphGetNodes(g, nodes.data(), &n));
  int64_t k = 0;
  for (auto& nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

extern "C" exp_status exp_ccsd_iterate(exp_ctx* x, int n_iter, exp_iter_info* info, int* converged) {
  API_BEGIN
  if (!x) throw ExpError{EXP_EINVAL, "null context"};
  Ctx& c = x->c;
  if (converged) *converged = 0;
  if (!c.have_integrals) throw ExpError{EXP_ESTATE, "exp_init_integrals must come first"};
  if (n_iter < 0) throw ExpError{EXP_EINVAL, "n_iter < 0"};
  if (!c.guessed) {
    if (c.cfg.guess == EXP_GUESS_MP2) ccsd_guess(c);
    else throw ExpError{EXP_ESTATE, "guess=USER needs exp_set_amplitudes first"};
    c.guessed = true;
  }
  bool all_conv = false;
  for (int it = 0; it < n_iter; ++it) {
    if (c.iter_done >= c.cfg.max_iter) return EXP_ENOTCONV;
    CK(cudaEventRecord(c.ev0, c.stream));
    if (c.graph) {
      CK(cudaGraphLaunch(c.graph, c.stream));
      c.launches += c.graph_kernels;
    } else {
      const bool capture = c.iter_done >= 1 && c.stream != nullptr && !c.profile;
      if (capture) {
        CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = c.launches;
        try {
          ccsd_iteration(c);
        } catch (...) {
          cudaGraph_t g;
          cudaStreamEndCapture(c.stream, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        cudaGraph_t g;
        CK(cudaStreamEndCapture(c.stream, &g));
        CK(cudaGraphInstantiate(&c.graph, g, 0));
        c.graph_kernels = count_kernel_nodes(g);
        CK(cudaGraphDestroy(g));
        c.launches = before + c.graph_kernels;
        CK(cudaGraphLaunch(c.graph, c.stream));
      } else {
        ccsd_iteration(c);
      }
    }
    CK(cudaEventRecord(c.ev1, c.stream));
    CK(cudaMemcpyAsync(c.h_stats, c.d_stats, sizeof(double) * 8 * c.ninst, cudaMemcpyDeviceToHost, c.stream));
    std::vector<int> st(4 * c.ninst);
    CK(cudaMemcpyAsync(st.data(), c.d_diis_state, sizeof(int) * 4 * c.ninst, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    c.iter_done++;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c.ev0, c.ev1));
    double mdt = 0.0;
    int nconv = 0, nfail = 0;
    for (int k = 0; k < c.ninst; ++k) {
      if (st[k * 4 + 2] == 1) ++nconv;
      else if (st[k * 4 + 2] == 2) ++nfail;
      else mdt = std::max(mdt, c.h_stats[k * 8 + 0]);
    }
    if (info) {
      info[it].e_re = c.h_stats[1];
      info[it].e_im = c.h_stats[2];
      info[it].max_dt = mdt;
      info[it].diis_n = int(c.h_stats[3]);
      info[it].n_converged = nconv;
      info[it].ms = ms;
    }
    if (c.d_emu_err) {
      int err = 0;
      CK(cudaMemcpy(&err, c.d_emu_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (err) throw ExpError{EXP_ETIMEOUT, "emulated GEMM: a bounded device wait gave up"};
    }
    c.n_failed = nfail;
    if (nconv + nfail == c.ninst) { all_conv = nfail == 0; break; }
  }
  if (converged) *converged = all_conv ? 1 : 0;
  if (c.n_failed) throw ExpError{EXP_ENUMERIC, std::to_string(c.n_failed) + " instance(s) diverged (NaN/Inf)"};
  if (!all_conv && c.iter_done >= c.cfg.max_iter) return EXP_ENOTCONV;
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_instance_state(exp_ctx* x, int inst, int* state) {
  API_BEGIN
  if (!x || !state) throw ExpError{EXP_EINVAL, "null argument"};
  Ctx& c = x->c;
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  int st[4];
  CK(cudaMemcpyAsync(st, c.d_diis_state + 4 * inst, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  *state = st[2];
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_energy(exp_ctx* x, int inst, double* e_re, double* e_im) {
  API_BEGIN
  if (!x) throw ExpError{EXP_EINVAL, "null context"};
  Ctx& c = x->c;
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  if (!c.guessed) throw ExpError{EXP_ESTATE, "no amplitudes yet"};
  double s[8];
  CK(cudaMemcpyAsync(s, c.d_stats + 8 * inst, sizeof(s), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  if (e_re) *e_re = s[1];
  if (e_im) *e_im = s[2];
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_fs_sector_0h1p(exp_ctx* x, int inst, double* heff, double* eig_re, double* eig_im,
                                         int* n_iter) {
  API_BEGIN
  if (!x) throw ExpError{EXP_EINVAL, "null context"};
  return fs_entry(x->c, inst, heff, eig_re, eig_im, n_iter);
  API_END(x)
}

extern "C" exp_status exp_fs_sector_0h2p(exp_ctx* x, int inst, double* heff, double* eig_re, double* eig_im,
                                         int* n_iter) {
  API_BEGIN
  if (!x) throw ExpError{EXP_EINVAL, "null context"};
  return fs2_entry(x->c, inst, heff, eig_re, eig_im, n_iter);
  API_END(x)
}

extern "C" exp_status exp_get_amplitudes(exp_ctx* x, int inst, void* t1, void* t2) {
  API_BEGIN
  if (!x || !t1 || !t2) throw ExpError{EXP_EINVAL, "null argument"};
  Ctx& c = x->c;
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  ccsd_dense_io(c, inst, (cplx*)t1, (cplx*)t2, true);
  CK(cudaStreamSynchronize(c.stream));
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_set_amplitudes(exp_ctx* x, int inst, const void* t1, const void* t2) {
  API_BEGIN
  if (!x || !t1 || !t2) throw ExpError{EXP_EINVAL, "null argument"};
  Ctx& c = x->c;
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  if (!c.have_integrals) throw ExpError{EXP_ESTATE, "exp_init_integrals must come first"};
  if (!c.guessed) {
    // other instances start from the MP2 guess
    ccsd_guess(c);
    c.guessed = true;
  }
  ccsd_dense_io(c, inst, (cplx*)t1, (cplx*)t2, false);
  ccsd_mark_guessed(c);
  CK(cudaStreamSynchronize(c.stream));
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_ccsd_t(exp_ctx* x, int inst, int block, exp_t3_info* info, double* per_triple) {
  API_BEGIN
  if (!x) throw ExpError{EXP_EINVAL, "null context"};
  ccsd_t(x->c, inst, block, info, per_triple);
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_work_per_iteration(const exp_ctx* x, double* macs) {
  API_BEGIN
  if (!x || !macs) throw ExpError{EXP_EINVAL, "null argument"};
  const Ctx& c = x->c;
  if (c.plans.empty()) throw ExpError{EXP_ESTATE, "no iteration planned yet"};
  double s = 0;
  for (auto& kv : c.plans) s += double(kv.second->g.flops_mac);
  *macs = s * c.ninst;
  return EXP_OK;
  API_END(const_cast<exp_ctx*>(x))
}

extern "C" exp_status exp_profile_top(exp_ctx* x, int reps, char* name, int name_len, double* ms,
                                      double* macs) {
  API_BEGIN
  if (!x || reps < 1) throw ExpError{EXP_EINVAL, "bad argument"};
  Ctx& c = x->c;
  if (c.plans.empty()) throw ExpError{EXP_ESTATE, "no iteration planned yet"};
  const std::string want = (name && name_len > 0) ? std::string(name, strnlen(name, size_t(name_len))) : "";
  const std::string* best = nullptr;
  EinsumPlan* P = nullptr;
  for (auto& kv : c.plans) {
    if (!want.empty()) {
      if (kv.first == want) { P = kv.second.get(); best = &kv.first; }
    } else if (!P || kv.second->g.flops_mac > P->g.flops_mac) {
      P = kv.second.get();
      best = &kv.first;
    }
  }
  if (!P) throw ExpError{EXP_EINVAL, "no contraction named " + want};
  Tensor* Cg = P->permC ? &P->C2 : nullptr;
  cplx* cd = Cg ? Cg->d : (P->gemm_out ? P->gemm_out : nullptr);
  int64_t cis = Cg ? Cg->is : P->gemm_out_is;
  if (!cd) throw ExpError{EXP_ESTATE, "contraction output unknown"};
  // per-iteration operand slices share one region: make them this product's again
  if (P->emulate) emu_run(c, P->emu, P->g, P->A->d, P->B->d, cd, P->A->is, P->B->is, cis, P->alpha, P->gemm_beta);
  CK(cudaStreamSynchronize(c.stream));
  CK(cudaEventRecord(c.ev0, c.stream));
  for (int r = 0; r < reps; ++r) {
    if (P->emulate)
      emu_run(c, P->emu, P->g, P->A->d, P->B->d, cd, P->A->is, P->B->is, cis, P->alpha, P->gemm_beta, true);
    else if (P->ds)
      launch_gemm_ds(c, P->g, P->A->d, P->B->d, cd, P->A->is, P->B->is, cis, P->alpha, P->gemm_beta);
    else
      launch_gemm_fp64(c, P->g, P->A->d, P->B->d, cd, P->A->is, P->B->is, cis, P->alpha, P->gemm_beta);
  }
  CK(cudaEventRecord(c.ev1, c.stream));
  CK(cudaEventSynchronize(c.ev1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, c.ev0, c.ev1));
  if (ms) *ms = double(t) / reps;
  if (macs) *macs = double(P->g.flops_mac) * c.ninst;
  if (name && name_len > 0) {
    strncpy(name, best->c_str(), size_t(name_len - 1));
    name[name_len - 1] = 0;
  }
  return EXP_OK;
  API_END(x)
}

extern "C" exp_status exp_zgemm(const exp_allocator* alloc, void* stream, int precision, int n_slices, int M,
                                int N, int K, const void* A, const void* B, void* C, double are, double aim,
                                int beta) {
  Ctx c;
  API_BEGIN
  if (!alloc || !alloc->alloc || !alloc->free || !A || !B || !C) throw ExpError{EXP_EINVAL, "null argument"};
  if (M < 1 || N < 1 || K < 0) throw ExpError{EXP_EINVAL, "bad GEMM shape"};
  if (precision != EXP_FP64 && precision != EXP_EMU_BF16 && precision != EXP_EMU_DS)
    throw ExpError{EXP_EINVAL, "bad precision"};
  if (precision == EXP_EMU_BF16 && (n_slices < 3 || n_slices > 6)) throw ExpError{EXP_EINVAL, "n_slices must be in 3..6"};
  if (precision == EXP_EMU_DS && K > 16) throw ExpError{EXP_EINVAL, "double-single product: K above 16"};
  if (precision == EXP_EMU_BF16 && K > EMU_MAX_K) throw ExpError{EXP_EINVAL, "emulated GEMM: K above 2^26"};
  c.alloc = *alloc;
  c.stream = (cudaStream_t)stream;
  c.cfg.precision = precision == EXP_EMU_DS ? EXP_EMU_BF16 : precision;
  c.cfg.n_slices = n_slices;
  c.autotune = false;  // a one-off product: nothing to amortise a tuning pass over
  c.ninst = 1;
  c.G = 1;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev));
  // a rank-2 "tensor" per operand: one block, rows x cols
  Layout LA, LB, LC;
  LA.G = LB.G = LC.G = 1;
  LA.rows = {M}; LA.cols = {K}; LA.blk_off = {0}; LA.size = int64_t(M) * K;
  LB.rows = {K}; LB.cols = {N}; LB.blk_off = {0}; LB.size = int64_t(K) * N;
  LC.rows = {M}; LC.cols = {N}; LC.blk_off = {0}; LC.size = int64_t(M) * N;
  GemmPlan g = make_gemm_plan(c, LA, LB, LC);
  const cplx alpha = make_double2(are, aim);
  if (precision == EXP_EMU_DS && K > 0) {
    ds_prepare(c, g);
    launch_gemm_ds(c, g, (const cplx*)A, (const cplx*)B, (cplx*)C, LA.size, LB.size, LC.size, alpha, beta != 0);
  } else if (precision == EXP_EMU_BF16 && K > 0) {
    Tensor TA, TB;
    TA.L = LA; TA.d = (cplx*)A; TA.is = LA.size;
    TB.L = LB; TB.d = (cplx*)B; TB.is = LB.size;
    EmuPlan* ep = emu_plan(c, g, &TA, &TB, false, false, true, "");
    emu_run(c, ep, g, (const cplx*)A, (const cplx*)B, (cplx*)C, LA.size, LB.size, LC.size, alpha, beta != 0);
  } else {
    launch_gemm_fp64(c, g, (const cplx*)A, (const cplx*)B, (cplx*)C, LA.size, LB.size, LC.size, alpha, beta != 0);
  }
  CK(cudaStreamSynchronize(c.stream));
  int err = 0;
  if (c.d_emu_err) CK(cudaMemcpy(&err, c.d_emu_err, sizeof(int), cudaMemcpyDeviceToHost));
  emu_release(c);
  c.dfree_all();
  if (err) throw ExpError{EXP_ETIMEOUT, "emulated GEMM: a bounded device wait gave up"};
  return EXP_OK;
  }
  catch (const ExpError& e) {
    g_err = e.msg;
    cudaStreamSynchronize(c.stream);
    emu_release(c);
    c.dfree_all();
    return e.s;
  }
  catch (const CudaError& e) {
    g_err = std::string(e.where) + ": " + cudaGetErrorString(e.e);
    cudaStreamSynchronize(c.stream);
    emu_release(c);
    c.dfree_all();
    return EXP_ECUDA;
  }
}

// Pade [L/M] fit through m points, E(0) = a0: unknowns (a0..aL, b1..bM), rows
// a0 + a1 x + ... + aL x^L - E (b1 x + ... + bM x^M) = E, solved in the least-squares
// sense (exactly when m = L + M + 1) by complex Householder QR and back substitution
// (the rows are Vandermonde-like, so the normal equations would square their condition).
extern "C" exp_status exp_pade_zero(int m, const double* x, const double* values, int L, int M, double* out) {
  g_err.clear();
  if (!x || !values || !out || L < 0 || M < 0 || m > 64 || m < L + M + 1) {
    g_err = "exp_pade_zero: need L, M >= 0 and L + M + 1 <= m <= 64 points";
    return EXP_EINVAL;
  }
  typedef std::complex<double> Z;
  const int nu = L + 1 + M;
  std::vector<Z> A(size_t(m) * nu), e(m);
  auto a = [&](int r, int c) -> Z& { return A[size_t(r) * nu + c]; };
  for (int k = 0; k < m; ++k) {
    e[k] = Z(values[2 * k], values[2 * k + 1]);
    double p = 1.0;
    for (int j = 0; j <= L; ++j, p *= x[k]) a(k, j) = p;
    p = x[k];
    for (int j = 1; j <= M; ++j, p *= x[k]) a(k, L + j) = -e[k] * p;
  }
  double amax = 0.0;
  for (auto& v : A) amax = std::max(amax, std::abs(v));
  // Householder: for column c, v = x + e^{i arg x0} |x| e1 over rows c..m-1; apply to A and e
  for (int c = 0; c < nu; ++c) {
    double nrm = 0.0;
    for (int r = c; r < m; ++r) nrm += std::norm(a(r, c));
    nrm = std::sqrt(nrm);
    if (!(nrm > 1e-15 * amax)) {
      g_err = "exp_pade_zero: singular system";
      return EXP_EINVAL;
    }
    const Z x0 = a(c, c);
    const Z ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : Z(1.0);
    std::vector<Z> v(m - c);
    for (int r = c; r < m; ++r) v[r - c] = a(r, c);
    v[0] += ph * nrm;
    double vn = 0.0;
    for (auto& q : v) vn += std::norm(q);
    for (int cc = c; cc < nu; ++cc) {  // A <- (I - 2 v v^H / v^H v) A
      Z d = 0.0;
      for (int r = c; r < m; ++r) d += std::conj(v[r - c]) * a(r, cc);
      d *= 2.0 / vn;
      for (int r = c; r < m; ++r) a(r, cc) -= d * v[r - c];
    }
    Z d = 0.0;
    for (int r = c; r < m; ++r) d += std::conj(v[r - c]) * e[r];
    d *= 2.0 / vn;
    for (int r = c; r < m; ++r) e[r] -= d * v[r - c];
  }
  std::vector<Z> coef(nu);
  for (int i = nu - 1; i >= 0; --i) {
    Z acc = e[i];
    for (int j = i + 1; j < nu; ++j) acc -= a(i, j) * coef[j];
    coef[i] = acc / a(i, i);
  }
  out[0] = coef[0].real();
  out[1] = coef[0].imag();
  return EXP_OK;
}

extern "C" int64_t exp_kernel_launches(const exp_ctx* x) { return x ? x->c.launches : 0; }

extern "C" const char* exp_last_error(const exp_ctx* x) {
  if (x && !x->c.err.empty()) return x->c.err.c_str();
  return g_err.c_str();
}
