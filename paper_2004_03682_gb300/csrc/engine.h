// Internal engine of libexpgb: symmetry-blocked tensors (DPD, Sec. II.C),
// permute / contract planning (the TTGT decomposition of Sec. II.B) and the
// context that owns device memory.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/exp.h"

typedef double2 cplx;  // (re, im)

#define EXP_MAX_RANK 4
#define EXP_MAX_TERMS 4
#define EXP_MAX_G 16
#define EXP_MAX_DIIS 8
#define EXP_CHUNK 4096  // elements per work chunk of a sub-block task (generators, permutes, tau)

// Spinor spaces.  Global spinor index: occupied 0..o-1, virtual o..o+v-1.
enum SpaceId { SP_OCC = 0, SP_VIRT = 1, SP_COUNT = 2 };

struct Space {
  int n = 0;
  std::vector<int> cnt;   // [G] spinors per irrep
  std::vector<int> off;   // [G] first local index of each irrep
  int gbase = 0;          // global index of local index 0
};

// A rank-r tensor stored as G dense matrices ("blocks"): block g has row
// compound = the first nrow slots with signed irrep sum g, column compound =
// the remaining slots with signed irrep sum -g (so every stored element obeys
// sum_k sign_k * irrep_k = 0 mod G).  Inside a block, row (column) tuples of
// slot irreps are enumerated lexicographically, each tuple a dense row-major
// sub-block.  sign +1 = created (upper) index, -1 = annihilated (lower).
struct Layout {
  int rank = 0;
  int sp[EXP_MAX_RANK] = {0, 0, 0, 0};
  int sg[EXP_MAX_RANK] = {1, 1, 1, 1};
  int nrow = 0;
  int G = 1;
  std::vector<int64_t> blk_off, rows, cols;  // [G]
  std::vector<int64_t> rtup, ctup;           // offsets of row / column tuples
  int64_t size = 0;                          // elements per instance

  std::string key() const;
};

// One dense sub-block (an allowed tuple of slot irreps) in a layout.
struct SubBlock {
  int irr[EXP_MAX_RANK];
  int n[EXP_MAX_RANK];
  int64_t base;
  int64_t st[EXP_MAX_RANK];
  int64_t count;
};

// Device task records ------------------------------------------------------
struct PermTask {
  int64_t dst;
  int64_t dst_st[4];
  int64_t src[EXP_MAX_TERMS];
  int64_t src_st[EXP_MAX_TERMS][4];
  int32_t n[4];
  int64_t count;     // elements, < 2^31
  uint32_t mg[4];    // division by n[d] as a multiply-high: see udiv_magic
  uint32_t ml[4];
  int32_t tri;       // bit 0: only elements i0 < i1, bit 1: only i2 < i3 (diagonal blocks
  int32_t pad_;      // of a canonical-pairs destination)
};

// q = floor(x / d) for 32-bit x as (t + ((x - t) >> 1)) >> (l - 1), t = umulhi(m, x),
// with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 (l = 0: q = x); the
// round-up method of Granlund and Montgomery (PLDI 1994).
inline void udiv_magic(uint32_t d, uint32_t& m, uint32_t& l) {
  l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
}

struct ChunkRef {
  int32_t task;
  int32_t pad;
  int64_t start;
};

struct GemmProb {  // one block of a grouped GEMM: C[MxN] (+)= alpha A[MxK] B[KxN], row-major
  int64_t a, b, c;  // element offsets inside the per-instance tensors
  int64_t ws;       // split-K partials offset in the plan's scratch (ksplit > 1)
  int32_t M, N, K;
  int32_t tile0;    // first tile index of this problem
  int32_t tiles_n;  // tiles along N
  int32_t tiles_m;
  int32_t ksplit;   // K ranges computed by separate CTAs, summed in fixed order
  int32_t kchunk;   // K per split (multiple of 8)
};

struct GenTask {  // integral generator: one sub-block
  int64_t base;
  int64_t st[4];
  int32_t n[4];
  int32_t g0[4];   // global spinor index of local index 0 of each slot
  int64_t count;
};

struct Ctx;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Scratch shared by the contractions of an iteration: each contraction's transient
// buffers (permuted operands, GEMM output, operand slices) live only during its own
// call, and the calls run in stream order, so they share one region per kind.
struct Arena {
  void* base = nullptr;
  size_t bytes = 0;
};

struct Tensor {
  Layout L;
  cplx* d = nullptr;  // instance k at d + k * is
  int64_t is = 0;     // instance stride in elements (>= L.size)
  // antisymmetric in slots (0, 1) and in (2, 3): while Ctx::canon_pairs is set, writes
  // into this tensor cover only the canonical entries (p < q in both pairs)
  bool pair_canon = false;
};

// Integral reference: V(p,q,r,s) with the spaces of its four arguments.
struct IntRef {
  int sp[4];
};

struct Operand {
  const Tensor* t = nullptr;   // either a tensor ...
  const IntRef* v = nullptr;   // ... or an integral class
  const char* labels = nullptr;  // one label per storage slot (tensor) or per V argument
};

struct PermPlan {
  PermTask* d_tasks = nullptr;
  ChunkRef* d_chunks = nullptr;
  int n_chunks = 0;
  int n_terms = 1;
};

struct GemmPlan {
  GemmProb* d_probs = nullptr;
  int n_probs = 0;
  int n_tiles = 0;
  int tm = 64, tn = 64;      // FP64 tile shape (16 or 64 each)
  cplx* d_ws = nullptr;      // split-K partials, ws_is elements per instance
  int64_t ws_is = 0;
  int64_t red_elems = 0;     // output elements of split problems (per instance)
  int64_t flops_mac = 0;  // complex MACs per instance
  int64_t dot_outputs = 0;  // > 0: run as one warp per output element (k_gemm_dot), this many outputs
  std::vector<GemmProb> h_probs;
  GemmProb* d_ds = nullptr;  // double-single SIMT tiles (k_gemm_ds), set by ds_prepare
  int ds_tiles = 0;
};

struct EmuPlan;  // emulated-GEMM plan (gemm_emu.cu)

struct EinsumPlan {
  // operand preparation
  bool permA = false, permB = false, permC = false;
  Tensor A2, B2, C2;  // permuted operands / GEMM output (views into scratch or cache)
  const Tensor* A = nullptr;
  const Tensor* B = nullptr;
  PermPlan pA, pB, pC;
  PermPlan pCc;  // pC restricted to the canonical entries (destination marked pair_canon)
  GemmPlan g;
  cplx alpha;
  cplx cterms[EXP_MAX_TERMS];
  bool gemm_beta = false;
  cplx* gemm_out = nullptr;  // GEMM output when it writes the destination directly
  int64_t gemm_out_is = 0;
  bool emulate = false;
  bool ds = false;  // short K under the emulated precision: double-single SIMT product
  bool swapped = false;  // operands exchanged at planning (C^T = B^T A^T); every call swaps them too
  int64_t offA2 = 0, offB2 = 0, offC2 = 0;  // element offsets of A2 / B2 / C2 in the operand arena
  EmuPlan* emu = nullptr;
  size_t scratch_bytes = 0;
};

int64_t layout_count(const Layout& L, const std::vector<Space>& spaces);

// Kernels (tensor.cu) --------------------------------------------------------
void launch_permute(Ctx& c, const PermPlan& p, cplx* dst, const cplx* src, int64_t dst_is,
                    int64_t src_is, const cplx* coef, bool accumulate, bool conj_src);
void launch_generate(Ctx& c, cplx* dst, int64_t inst_stride, const GenTask* d_tasks,
                     const ChunkRef* d_chunks, int n_chunks, const int map[4]);
void launch_fill_denom(Ctx& c, double* dst, int64_t inst_stride, const GenTask* d_tasks,
                       const ChunkRef* d_chunks, int n_chunks, int nslots, const int sgn[4],
                       const double* eps);
void launch_tau(Ctx& c, cplx* dst, int64_t dst_is, const cplx* t2, const cplx* t1,
                int64_t t_is, const int32_t* t1_index, const GenTask* d_tasks,
                const ChunkRef* d_chunks, int n_chunks, double c0, double c1, double c2);
void launch_tau3(Ctx& c, cplx* tau, cplx* taut, cplx* zeta, int64_t dst_is, const cplx* t2, const cplx* t1,
                 int64_t t_is, const int32_t* t1_index, const GenTask* d_tasks, const ChunkRef* d_chunks,
                 int n_chunks);
void launch_gemm_fp64(Ctx& c, const GemmPlan& g, const cplx* A, const cplx* B, cplx* C,
                      int64_t a_is, int64_t b_is, int64_t c_is, cplx alpha, bool beta);
// double-single SIMT product for short contractions (every K <= 16) under the
// emulated precision: ds_wanted decides, ds_prepare builds its tile list once
bool ds_wanted(Ctx& c, const GemmPlan& g);
void ds_prepare(Ctx& c, GemmPlan& g);
void launch_gemm_ds(Ctx& c, const GemmPlan& g, const cplx* A, const cplx* B, cplx* C, int64_t a_is,
                    int64_t b_is, int64_t c_is, cplx alpha, bool beta);

// Context -------------------------------------------------------------------
struct Ctx {
  exp_config cfg{};
  exp_allocator alloc{};
  cudaStream_t stream = nullptr;
  std::string err;
  int G = 1, no = 0, nv = 0, ninst = 1;
  std::vector<Space> spaces;
  int sm_count = 0;
  int64_t launches = 0;

  // per-instance device data
  double* d_eps = nullptr;        // [ninst][n]
  uint64_t* d_seed = nullptr;     // [ninst]
  double* d_scale = nullptr;      // [ninst]
  std::vector<double> h_scale;
  bool have_integrals = false;

  // amplitude vector T = [t1 | t2] per instance and its companions
  Tensor t1, t2, r1, r2;           // views into the vectors below
  int64_t n1 = 0, n2 = 0, namp = 0;
  cplx* d_T = nullptr;             // [ninst][namp] current amplitudes
  cplx* d_R = nullptr;             // [ninst][namp] right-hand sides
  double* d_D = nullptr;           // [ninst][namp] denominators
  cplx* d_diis_t = nullptr;        // [ninst][diis][namp]
  cplx* d_diis_e = nullptr;        // [ninst][diis][namp]
  double* d_diis_B = nullptr;      // [ninst][diis][diis]
  int* d_diis_state = nullptr;     // [ninst][4]: count, head, converged, pad
  double* d_stats = nullptr;       // [ninst][4]: max_dt, e_re, e_im, diis_n
  double* h_stats = nullptr;       // pinned host mirror
  int iter_done = 0;
  int n_failed = 0;  // instances frozen after NaN/Inf
  bool guessed = false;

  // caches
  std::map<std::string, std::unique_ptr<Tensor>> int_cache;   // integral layouts
  struct IntMeta {
    int vsp[4], arg[4];  // spaces of the V arguments; storage slot k holds V argument arg[k]
    const Tensor* t;
  };
  std::vector<IntMeta> int_list;  // the cached layouts, for deriving related ones
  bool integrals_scaled = false;  // the MP2 scale is final (set by exp_init_integrals)
  bool canon_pairs = false;       // writes into pair_canon tensors: canonical entries only
  std::map<std::string, PermPlan> perm_cache;
  std::map<std::string, std::unique_ptr<EinsumPlan>> plans;   // by call-site key
  std::vector<DevBuf> owned;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;

  // CCSD work tensors (created on first iteration)
  std::map<std::string, std::unique_ptr<Tensor>> work;

  // CUDA graph of one iteration
  cudaGraphExec_t graph = nullptr;
  int64_t graph_kernels = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool profile = false;  // EXP_PROFILE=1: eager iterations, per-contraction timing on stderr
  bool autotune = true;  // time candidate work decompositions of each emulated product once
  double force_ksplit_mult = -1.0;  // >= 0 with autotune off: this K-split multiplier
  int force_group_rows = 0;         // > 0 with autotune off: this work-order group size
  cudaEvent_t pev0 = nullptr, pev1 = nullptr;

  int* d_emu_err = nullptr;  // set by a bounded device wait that gave up
  // (0h,1p) sector: one non-interacting "ghost" occupied spinor per active virtual
  int no_real = 0, nact = 0, n_gen = 0;
  std::vector<int> act;        // active virtual local indices (config order)
  std::vector<int> occ_real;   // occupied local index -> real occupied index, -1 for a ghost
  std::vector<int> occ_ghost;  // occupied local index -> active slot, -1 for a real spinor
  int* d_genmap = nullptr;     // global spinor index -> generator index (-1: ghost), or null
  int* d_occreal = nullptr;    // device copy of occ_real
  double* d_eps_fs = nullptr;  // [ninst][n] orbital energies with ghost x <- eps of active x
  void* fs_state = nullptr;

  // emulation and driver state
  void* emu_state = nullptr;
  void* packed_state = nullptr;  // packed particle-particle ladder (packed.cu)
  void* ccsd_state = nullptr;

  Arena op_arena;     // permuted operands and GEMM outputs of one contraction
  Arena slice_arena;  // per-iteration operand slices of one emulated product

  // pinned staging for stream-ordered uploads (upload_async): two halves used in turn,
  // each released by an event once the copies out of it have run
  struct Staging {
    uint8_t* host[2] = {nullptr, nullptr};
    size_t cap = 0, used = 0;
    int cur = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool pending[2] = {false, false};
  } stg;

  void* dalloc(size_t bytes);
  void dfree(void* p);
  void dfree_all();
};

// Helpers (engine.cu)
GemmPlan make_gemm_plan(Ctx& c, const Layout& A, const Layout& B, const Layout& C);
void build_layout(Layout& L, const std::vector<Space>& spaces, int G);
Layout make_layout(const std::vector<Space>& spaces, int G, int rank, const int* sp,
                   const int* sg, int nrow);
void enumerate_blocks(const Layout& L, const std::vector<Space>& spaces,
                      std::vector<SubBlock>& out);
Tensor* new_tensor(Ctx& c, const Layout& L, bool zero);
// grow an arena to at least `bytes` (only outside stream capture; synchronises the
// stream before the old region is released); returns its base
void* arena_reserve(Ctx& c, Arena& a, size_t bytes);
Tensor* work_tensor(Ctx& c, const std::string& name, const Layout& L);
const Tensor* integral(Ctx& c, const IntRef& v, const int perm[4], int nrow);
// the same layout derived from a cached member of its symmetry family, not cached:
// the caller releases it (c.dfree(t->d); delete t); nullptr when no member is cached
Tensor* integral_uncached(Ctx& c, const IntRef& v, const int perm[4], int nrow);
void gen_tasks(Ctx& c, const Layout& L, std::vector<GenTask>& tasks,
               std::vector<ChunkRef>& chunks);
void einsum(Ctx& c, const std::string& site, cplx alpha, Operand A, Operand B, Tensor& C,
            const char* clabels, bool accumulate,
            std::vector<std::pair<double, std::string>> terms = {});
void permute_into(Ctx& c, const std::string& site, Tensor& dst, const char* dlabels,
                  const Tensor& src, const char* slabels, bool accumulate,
                  std::vector<std::pair<double, std::string>> terms = {});
void upload(Ctx& c, void* dst, const void* src, size_t bytes);
// the same copy, stream-ordered: the host data are staged in pinned memory and the
// call returns at once (large copies fall back to upload)
void upload_async(Ctx& c, void* dst, const void* src, size_t bytes);
void staging_release(Ctx& c);

struct CudaError {
  cudaError_t e;
  const char* where;
};
struct ExpError {
  exp_status s;
  std::string msg;
};
#define CK(x)                                            \
  do {                                                   \
    cudaError_t _e = (x);                                \
    if (_e != cudaSuccess) throw CudaError{_e, #x};      \
  } while (0)
#define KCHECK(c)                                        \
  do {                                                   \
    (c).launches++;                                      \
    cudaError_t _e = cudaGetLastError();                 \
    if (_e != cudaSuccess) throw CudaError{_e, "launch"}; \
  } while (0)

struct exp_ctx {
  Ctx c;
};
