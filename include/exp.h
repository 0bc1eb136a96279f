/*
 * exp.h -- C ABI of libexpgb: the data-parallel hot path of relativistic
 * Fock-space coupled cluster (CCSD amplitude equations and the (0h,1p) sector)
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method (Oleynichenko, Zaitsevskii, Eliav, "Towards High Performance
 * Relativistic Electronic Structure Modelling: The EXP-T Program Package",
 * arXiv:2004.03682):
 *   - Hamiltonian in second-quantised form, Eq. (ham); V_pqrs = <pq||rs> is the
 *     coefficient of (1/4) {p+ q+ s r}; f = diag(eps) (Hartree-Fock spinors).
 *   - Amplitude equations t = D^-1 (V Omega - Omega (V Omega)_Cl), Eq. (amplitudes),
 *     with D the negated differences of H0 eigenvalues; sectors solved one after
 *     another, Eq. (sectors): (0h,0p) then (0h,1p).
 *   - Every diagram is evaluated as permute -> GEMM -> permute (the TTGT list of
 *     Sec. II.B) on symmetry-blocked tensors (DPD, Sec. II.C, Fig. "blocks"),
 *     with all blocks of one contraction in one grouped launch (Fig. "mult").
 *
 * Conventions for every entry point:
 *   - All host pointers are read during the call only (copied); nothing is
 *     retained.  Device memory is obtained only through the caller's
 *     exp_allocator, on the caller's CUDA stream; the library never calls
 *     cudaMalloc.  All device work is ordered on that stream.  An entry point
 *     that returns host values synchronises that stream (only).
 *   - No exception or abort crosses the ABI.  Every call returns an exp_status;
 *     exp_last_error() gives a one-line message for the last failure.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Complex numbers are (re, im) pairs of IEEE doubles.
 *
 * Environment variables read at exp_create (diagnostics and timing studies only; none
 * changes a result bit):
 *   EXP_PROFILE=1       iterations run eagerly (no CUDA graph), with per-contraction and
 *                       per-stage times and the (T) stage times on stderr;
 *   EXP_AUTOTUNE=0      keep the default work decomposition of the emulated products
 *                       instead of timing the candidates on their first run;
 *   EXP_KSPLIT_MULT=m   with EXP_AUTOTUNE=0: this K-split multiplier (0 = no split);
 *   EXP_GROUP_ROWS=g    with EXP_AUTOTUNE=0: g row tiles per group of the work order.
 * Split-K partials are exact integers added in 128 bits, so no decomposition changes a
 * bit of an emulated product.
 */
#ifndef EXPGB_EXP_H
#define EXPGB_EXP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EXP_OK = 0,
  EXP_EINVAL = 1,    /* bad argument, shape or label */
  EXP_ENOMEM = 2,    /* the allocator returned NULL */
  EXP_ECUDA = 3,     /* a CUDA runtime error (message in exp_last_error) */
  EXP_ENOTCONV = 4,  /* max_iter reached without convergence */
  EXP_ENUMERIC = 5,  /* NaN/Inf in the amplitudes */
  EXP_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
  EXP_ESTATE = 7     /* call order violated (e.g. 0h1p before converged 0h0p) */
} exp_status;

typedef struct exp_ctx exp_ctx;

/* Device memory provider.  alloc(bytes, user) returns a device pointer (256-byte
 * aligned) usable on the context's stream, or NULL; free(ptr, user) releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} exp_allocator;

/* EXP_EMU_DS (exp_zgemm only): double-single FP32 SIMT product, K <= 16 -- what the
 * EXP_EMU_BF16 contractions use when every block has K <= 16 (Sec. II.B step 3).
 * Each operand is carried as two FP32 numbers (48 bits); |x| < 2^-126 counts as 0 and
 * |x| >= 2^128 as infinite; error within about K 2^-47 of sum |a||b| per element. */
enum { EXP_FP64 = 0, EXP_EMU_BF16 = 1, EXP_EMU_DS = 2 };
enum { EXP_GUESS_MP2 = 0, EXP_GUESS_USER = 1 };

typedef struct {
  int n_inst;              /* independent same-sized instances solved together (>= 1) */
  int n_occ, n_virt;       /* occupied (hole) and virtual (particle) spinors */
  int n_irrep;             /* G: cyclic Abelian labels Z_G (1 = no symmetry) */
  const int32_t* irrep_occ;   /* [G] occupied spinors per irrep (shared by instances) */
  const int32_t* irrep_virt;  /* [G] virtual spinors per irrep */
  const double* eps_occ;      /* [n_inst * n_occ] orbital energies, ordered by irrep then energy */
  const double* eps_virt;     /* [n_inst * n_virt] */
  int precision;           /* EXP_FP64: all contractions in FP64.  EXP_EMU_BF16: the large
                              contractions as split-precision emulation of complex FP64 on
                              the BF16 tensor cores, those with every K <= 16 in double-single
                              FP32 arithmetic (update, DIIS, energy stay FP64). */
  int n_slices;            /* BF16 slices per FP64 operand in emulation (3..6) */
  int diis_dim;            /* Pulay DIIS subspace (0 = off, <= 8) */
  double conv_tol;         /* converged when max |t_new - t| < conv_tol */
  int max_iter;            /* per exp_ccsd_iterate sequence, counted from the guess */
  int guess;               /* EXP_GUESS_MP2 or EXP_GUESS_USER (amplitudes set by exp_set_amplitudes) */
  double emu_min_macs;     /* with EXP_EMU_BF16: contractions with fewer complex multiply-adds per
                              instance stay FP64 (0 = default) */
  int n_active;            /* (0h,1p) sector: number of active (valence) virtual spinors, 0 = none */
  const int32_t* active_virt; /* [n_active] their indices within the virtual space (config order),
                                 shared by all instances; NULL when n_active = 0 */
  double level_shift;      /* sigma >= 0: (0h,0p) update t <- t + (RHS - D t)/(D - sigma) (the same
                              fixed point; smaller steps for strongly coupled problems); 0 = the
                              plain update t <- RHS/D.  The (0h,1p) Bloch update divides by
                              D + sigma sign(D) the same way. */
  int packed;              /* 1: the particle-particle ladder sum_{c<d} <ab||cd> tau_ij^cd and the other
                              products over a tau pair on pair-packed operands (a<b, c<d, i<j per
                              pair irrep; <ab||cd> stored packed, a quarter of the full size), and
                              the update, DIIS vectors and energy on t1 plus the a<b, i<j entries of
                              t2 (same fixed point and DIIS matrix as full vectors); 0: full pair
                              compounds everywhere */
  int n_slices_major;      /* with EXP_EMU_BF16: BF16 slices (3..6; 0 = n_slices) for the products that
                              carry nearly all of the tensor work -- the particle-particle ladder
                              <ab||cd> tau_ij^cd, its W_abef companion X_amij = <am||ef> tau_ij^ef,
                              and the two ring products (t2 W_mbej and the t2 <mn||ef> term of
                              W_mbej).  Every other emulated product (the hole-hole ladder and
                              W_mnij, the F intermediates, the T1-equation terms, the t1- and
                              F-coupled T2 terms) takes n_slices: those form or apply
                              intermediates whose errors act on every amplitude alike and set the
                              energy's accuracy, at a small share of the work. */
  double denom_shift;      /* s >= 0: intruder-state denominator shift (Sec. II.A, after Eq. (sectors)):
                              every energy denominator D of the amplitude equations is replaced by
                              D~ = D - s (s / (s + |D|))^n ("dynamic": a near-zero or positive D moves
                              by about -s, one with |D| >> s hardly at all), in both sectors:
                              (0h,0p) D~ t = RHS(t) (guess V/D~), (0h,1p) rho + (D - D~) s = 0 stepped
                              with 1/D~.  The solution depends on s; exp_pade_zero extrapolates
                              results at several s to s = 0.  0 = the plain equations. */
  int denom_shift_n;       /* n >= 1, the attenuation power of the dynamic shift (ignored when s = 0) */
  int real_arith;          /* 1: real Hamiltonian, real arithmetic (the paper's real double groups, Sec. II.C,
                              Table tab:time): the integrals are the recipe's real part (the recipe on
                              Re A), and the emulated products run as real GEMMs (A' = Re A, one B row
                              per output column: a quarter of the complex tensor work); storage stays
                              complex with zero imaginary parts, the FP64 kernels unchanged.  0: complex. */
} exp_config;

/* Create a context: validates the config, builds the symmetry-blocked layouts
 * (Sec. II.C) and allocates amplitude/denominator/DIIS storage.  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  EINVAL on bad sizes (n_occ < 1,
 * n_virt < 1, G < 1, counts not summing to n_occ/n_virt, n_slices outside 3..6,
 * diis_dim > 8); ENOMEM when the allocator fails. */
exp_status exp_create(const exp_config* cfg, const exp_allocator* alloc, void* stream,
                      exp_ctx** out);
void exp_destroy(exp_ctx* ctx);

/* Step I of the flowchart (Sec. II.B): generate the synthetic two-electron
 * integrals of every instance directly in the blocked layouts the contractions
 * read.  V follows the seeded recipe: A_pqrs complex Gaussian from Philox4x32-10
 * at counter (idx, 0, 0), key seed; V = A - A(qp) - A(sr) + A(qp,sr);
 * V <- (V + conj V_rspq)/2; V_pqrs = 0 unless G_p + G_q - G_r - G_s = 0 mod G;
 * V <- s V with s = 0.05 / max|V_abij / D_ij^ab|, times scale_mult[k].
 * seeds: [n_inst] host.  scale_mult: [n_inst] host or NULL (= 1).  scale_out:
 * [n_inst] host or NULL, receives each applied s * scale_mult. */
exp_status exp_init_integrals(exp_ctx* ctx, const uint64_t* seeds, const double* scale_mult,
                              double* scale_out);

/* Per-iteration record (host). */
typedef struct {
  double e_re, e_im;   /* E(t_new) of instance 0 */
  double max_dt;       /* max over instances of max |t_new - t| */
  int diis_n;          /* vectors in the DIIS subspace (instance 0) */
  int n_converged;     /* instances converged after this iteration */
  double ms;           /* device time of the iteration (CUDA events) */
} exp_iter_info;

/* Steps II-IV for the (0h,0p) sector: iterate the CCSD amplitude equations
 * (Eq. (amplitudes) with T = T1 + T2) from the guess (first call) or from the
 * current amplitudes.  One iteration: build tau, the F/W intermediates and all
 * T1/T2 diagrams (grouped permute + contraction launches), t_new = RHS/D,
 * residual max|t_new - t|, E(t_new), DIIS extrapolation.  Runs at most n_iter
 * iterations, stopping early when every instance has converged (residual below
 * conv_tol) or failed.  An instance whose amplitudes turn NaN/Inf is frozen as
 * failed and the others go on; the call then returns ENUMERIC.  info: host array
 * of n_iter records or NULL.  *converged (host, nullable) = 1 when all instances
 * converged.  Returns ENOTCONV once max_iter iterations have run in total without
 * convergence, ESTATE before exp_init_integrals. */
exp_status exp_ccsd_iterate(exp_ctx* ctx, int n_iter, exp_iter_info* info, int* converged);

/* State of instance `inst`: 0 iterating, 1 converged, 2 failed (NaN/Inf).  Synchronises. */
exp_status exp_instance_state(exp_ctx* ctx, int inst, int* state);

/* Correlation energy of instance `inst` for the current amplitudes (E of the last
 * t_new; the MP2 energy before any iteration), in hartree.  Synchronises. */
exp_status exp_energy(exp_ctx* ctx, int inst, double* e_re, double* e_im);

/* Steps II-V for the (0h,1p) sector (Eq. (sectors); H_eff = (H Omega)_Cl, Sec. II.A;
 * flowchart step V, Sec. II.B): with the (0h,0p) amplitudes T converged, solve the
 * Bloch equation Q Hbar (P + S) = S H_eff, H_eff = P Hbar (P + S), for the
 * one-valence-particle amplitudes s_x^a, s_xj^ab of the configured active spinors
 * (the contractions of Eq. (eq:contraction) and its companions, all through the
 * same grouped permute/GEMM launches), iterating s <- s + (Q Hbar (P+S) - S H_eff)/D
 * with D_x^a = e_x - e_a, D_xj^ab = e_x + e_j - e_a - e_b and DIIS, then
 * diagonalise H_eff per irrep block (FP64 shifted QR on the device).  Runs the
 * iteration for all instances on the first call (conv_tol, max_iter and diis_dim
 * of the config), then reports instance `inst`: heff (host, n_active^2 (re, im)
 * pairs, row y = active y, column x; nullable), eig_re / eig_im (host, n_active,
 * sorted by real part, then imaginary part), *n_iter (nullable).  ESTATE unless
 * every instance's (0h,0p) iteration has converged and n_active > 0; ENOTCONV if
 * the Bloch iteration did not converge within max_iter. */
exp_status exp_fs_sector_0h1p(exp_ctx* ctx, int inst, double* heff, double* eig_re, double* eig_im,
                              int* n_iter);

/* Step V for the (0h,2p) sector (Eq. (sectors), the next sector after (0h,1p); the
 * paper's KCs2+ -> KCs scheme reaches KCs through it): with T and the (0h,1p)
 * amplitudes converged and fixed (the (0h,1p) sector is run first when it has not
 * been), solve for the two-valence-particle amplitudes s_xy^ab (x < y active, a < b
 * not both active) the Bloch equation projected on the two-particle determinants,
 *   Q Hbar Omega P = Q Omega P H_eff,   H_eff = P Hbar Omega P,   Omega = {exp(S1 + S2)},
 * in connected form: rho_xy^ab = [Hbar Omega]_conn - sum_z s_zy^ab H1_zx
 * - sum_w s_xw^ab H1_wy - 1/2 sum_zw tau_zw^ab H2_zw,xy (H1 the (0h,1p) H_eff, H2 the
 * connected two-particle part, tau_zw^ab = s_zw^ab + c_z^a c_w^b - c_z^b c_w^a with
 * c = P + S1), iterated s <- s + rho / (e_x + e_y - e_a - e_b) with DIIS through the same
 * grouped contraction launches; then H_eff = H1 (x) 1 + 1 (x) H1 + H2 on the pairs is
 * diagonalised per pair irrep on the device.  Reports instance `inst`: heff (host,
 * npair^2 (re, im), npair = n_active (n_active - 1) / 2; row = pair (z, w), column =
 * pair (x, y), pairs x < y in the order (0,1), (0,2), ..., (1,2), ... of the active
 * slots; nullable), eig_re / eig_im (host, npair, sorted by real then imaginary part:
 * double-attachment energies relative to the CCSD ground state), *n_iter (nullable).
 * ESTATE with fewer than two active spinors or when the (0h,1p) sector did not
 * converge; EINVAL when a pair-irrep block exceeds 32 pairs; ENOTCONV if the
 * (0h,2p) iteration did not converge within max_iter. */
exp_status exp_fs_sector_0h2p(exp_ctx* ctx, int inst, double* heff, double* eig_re, double* eig_im,
                              int* n_iter);

/* Zero-shift extrapolation of results computed with denominator shifts (Sec. II.A;
 * Sec. III.A: dynamic shifts with Pade extrapolation to the zero-shift limit): the
 * values E_k (m complex numbers, (re, im) pairs, host) at scales x_k (m doubles, host)
 * are fitted by E(x) = (a0 + a1 x + ... + aL x^L) / (1 + b1 x + ... + bM x^M) through the
 * linear conditions a0 + ... + aL x_k^L - E_k (b1 x_k + ... + bM x_k^M) = E_k (solved
 * exactly when m = L + M + 1, in least squares when m is larger, by Householder QR); *out (host, one
 * (re, im) pair) receives a0 = E(0).  With the dynamic shift of power n the natural
 * scale is x_k = s_k^(n+1) (the leading order of D - D~ for |D| >> s).  Host only, no
 * GPU work.  EINVAL if m < L + M + 1, m > 64, L < 0, M < 0 or the system is singular. */
exp_status exp_pade_zero(int m, const double* x, const double* values, int L, int M, double* out);

/* Copy amplitudes of instance `inst` between the context and caller device
 * buffers, dense layout: t1[i][a] (n_occ x n_virt), t2[i][j][a][b]; complex128,
 * spinor order as in the config.  Symmetry-forbidden elements read as 0 and are
 * ignored on write.  set_amplitudes also resets DIIS and the iteration count. */
exp_status exp_get_amplitudes(exp_ctx* ctx, int inst, void* t1_dev, void* t2_dev);
exp_status exp_set_amplitudes(exp_ctx* ctx, int inst, const void* t1_dev, const void* t2_dev);

/* Result of exp_ccsd_t. */
typedef struct {
  double e_re, e_im;     /* E(T), hartree */
  double ms;             /* device time of the call on the context stream (CUDA events) */
  double ms_products;    /* of which the product launches (the connected contractions) */
  double ms_energy;      /* of which the per-triple energy launches */
  double macs;           /* complex multiply-adds of the connected-triples contractions the
                            triples i<j<k need (the method's work) */
  double macs_run;       /* complex multiply-adds of the products launched (each (triple, pair
                            irrep) product covers exactly its three terms: equal to macs) */
  double x_elems;        /* complex elements of the products' outputs Y (one per triple, pair
                            irrep, virtual a and pair b<c; each read once by the energy kernel) */
  int64_t n_triples;     /* occupied triples i<j<k */
  int n_block_triples;   /* batches (the triples of one occupied block triple) processed */
  int block;             /* occupied spinors per block */
} exp_t3_info;

/* The perturbative triples correction (T) of CCSD(T) (the model list of Sec. III.A)
 * for instance `inst`, from the amplitudes the context holds (converged by
 * exp_ccsd_iterate, or set by exp_set_amplitudes), for the Hartree-Fock reference
 * of the synthetic Hamiltonian (f diagonal):
 *   c_ijk^abc = P(i/jk) P(a/bc) [ sum_e <bc||ei> t_jk^ae - sum_m <ma||jk> t_im^bc ],
 *   d_ijk^abc = P(i/jk) P(a/bc) t_i^a <bc||jk>,  P(p/qr) f = f - f(p<->q) - f(p<->r),
 *   E(T) = sum over i<j<k, a<b<c of conj(c + d) c / (e_i + e_j + e_k - e_a - e_b - e_c).
 * The connected contractions run as one product per triple and pair irrep of (b, c)
 * (the three terms' K concatenated), grouped per batch of triples, in the context's
 * precision (EXP_EMU_BF16: the BF16-sliced emulation with n_slices slices; EXP_FP64:
 * the FP64 kernel).  The permutations, the disconnected term, the
 * denominators and the energy terms run in FP64 under EXP_FP64 and in double-single
 * FP32 (about 48 bits) under EXP_EMU_BF16; the sums over elements and triples are FP64
 * in fixed order, so the result does not depend on the work
 * decomposition.  block: occupied spinors per block of the schedule (a batch is the
 * triples of one block triple; 0: the largest block size whose batch outputs fit the
 * scratch budget; a larger value than n_occ means n_occ); every block size gives the
 * same bits.  info (host, nullable) receives E(T)
 * and the work counts;
 * per_triple (host, nullable, 2 * n_triples doubles) receives each triple's
 * (re, im) energy at index C(k,3) + C(j,2) + i of its i<j<k (spinor order of the
 * config).  Needs about 16 GiB of scratch for a batch's product outputs at most, plus
 * dense t2 and <bc||jk> (n_occ^2 n_virt^2 each) and the fixed operands
 * (n_occ n_virt^2 (n_virt + n_occ) / (2 G)); the integrals <bc||ep> and <ma||qr> it
 * reads in a layout the context did not hold yet stay in the context's integral cache
 * (n_virt^3 n_occ / G and n_occ^3 n_virt / G complex elements per instance).
 * Synchronises.  ESTATE before
 * exp_init_integrals or before any amplitudes exist, and for a context with an
 * active space; EINVAL for inst out of range, block < 0 or more than 65535 virtual
 * spinors;
 * ETIMEOUT if a bounded wait of the emulated GEMM gave up. */
exp_status exp_ccsd_t(exp_ctx* ctx, int inst, int block, exp_t3_info* info, double* per_triple);

/* Algorithmic work of one (0h,0p) iteration, all instances: complex
 * multiply-adds of every contraction over the symmetry-allowed blocks (what the
 * grouped GEMMs execute).  Valid after the first iteration has been planned. */
exp_status exp_work_per_iteration(const exp_ctx* ctx, double* complex_macs);

/* Time one contraction on its own: `reps` launches of its grouped GEMM kernel on
 * the context stream between CUDA events (emulated: one full product first to put
 * its operand slices in place, then the tensor-core kernel alone; the slicing
 * passes and a split-K reduction are not timed).  `name` is in-out: on entry a
 * call-site name selects the contraction (EINVAL if there is none of that name), an
 * empty string selects the one with the most work; on return it holds the site
 * profiled (NUL-terminated, truncated to name_len).  Writes the mean milliseconds
 * per launch and its complex multiply-adds per launch.  Overwrites that
 * contraction's output buffer, which the next iteration recomputes. */
exp_status exp_profile_top(exp_ctx* ctx, int reps, char* name, int name_len, double* ms_per_launch,
                           double* complex_macs_per_launch);

/* One complex GEMM C = alpha A B (+ C if beta) on caller device buffers, with the
 * same kernels the contractions use (step 3 of the TTGT list, Sec. II.B):
 * precision EXP_FP64 (SIMT FP64), EXP_EMU_DS (double-single FP32 SIMT, K <= 16)
 * or EXP_EMU_BF16 (n_slices BF16 slices on the
 * tcgen05 tensor cores).  A: M x K, B: K x N, C: M x N, row-major complex128
 * (re, im doubles), 16-byte aligned.  Scratch (slices, exponents, split-K
 * partials) comes from `alloc` and is released before return.  Ordered on
 * `stream`; synchronises it.  EINVAL on M, N < 1, K < 0 or bad precision /
 * n_slices; ETIMEOUT if a bounded device wait gave up. */
exp_status exp_zgemm(const exp_allocator* alloc, void* stream, int precision, int n_slices, int M, int N, int K,
                     const void* A, const void* B, void* C, double alpha_re, double alpha_im, int beta);

/* Test hook of the bounded device waits (no counterpart in the paper; for tests of
 * the timeout path only).  Every wait inside the emulated tensor-core GEMM gives up
 * after a limit (2 s) and sets an error flag that the host reads (EXP_ETIMEOUT); the
 * kernel then waits, with the same limit, for its own copies in flight, releases its
 * tensor memory and returns, so the context stays usable.  exp_test_emu_wait sets that
 * limit to wait_ms (0 < wait_ms <= 2000) and, with skip_kblock >= 0, makes CTA 0 of
 * every later GEMM launch leave the slice copies of its k-block number skip_kblock
 * unissued, so the wait on that stage runs out with nothing in flight for it.
 * exp_test_emu_wait(-1, 2000) restores the normal behaviour.  Process-wide, for the
 * launches that follow on any thread.  EINVAL on arguments out of range. */
exp_status exp_test_emu_wait(int skip_kblock, double wait_ms);

/* Allocation-free complex GEMM (no counterpart in the paper: a library service).
 *
 * For callers that cannot allocate device memory when they need the product -
 * a host application that owns every allocation and hands this library only a
 * stream and its buffers, a pool whose budget is already spent, or a path where
 * a cudaMalloc would synchronise the device.  Computes C = alpha A B (+ C if
 * beta) with the BF16-sliced emulation of exp_zgemm (EXP_EMU_BF16, n_slices in
 * 3..6; same layouts: A M x K, B K x N, C M x N, row-major complex128 device
 * buffers, 16-byte aligned), and calls no allocator, cudaMalloc or cudaFree.
 *
 * Its scratch is one fixed array in the library's device memory, of
 * EXP_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
 * the process exits.  A problem whose scratch need exceeds it is rejected with
 * EXP_EINVAL before anything is launched (square problems fit up to about
 * M = N = K = 600 with n_slices = 5 or 6; K above 2^26 is refused before any size
 * is derived from it).
 * The first call on a device (and again after a new context replaces the device's
 * old one, e.g. after cudaDeviceReset) looks the array's address up with that
 * device current; make it before any stream capture.  Every call shares the array
 * and re-initialises what must start at a known value; calls whose GPU work can
 * overlap (different streams without ordering) race on it.  Synchronises
 * `stream`.  Errors: EINVAL, ECUDA (also when a CUDA error was already pending on
 * the calling thread; nothing is launched then), ETIMEOUT; message in
 * exp_noalloc_last_error().  On ECUDA or ETIMEOUT the contents of C are
 * unspecified. */
#define EXP_NOALLOC_SCRATCH_BYTES (48u << 20)
exp_status exp_zgemm_emu_noalloc(void* stream, int n_slices, int M, int N, int K, const void* A, const void* B,
                                 void* C, double alpha_re, double alpha_im, int beta);
const char* exp_noalloc_last_error(void);

/* Learned initial guess for T2 (no counterpart in the paper; a starting point for
 * the amplitude iteration, which alone decides the converged result).  A 3-layer
 * MLP of width 128 maps the features (|t_MP2|/0.05, -D_ij^ab/10,
 * |<ij||ab>|/max|<ij||ab>|) of every doubles amplitude to a complex multiplier:
 * t2 = (1 + y0 + i y1) <ab||ij>/D_ij^ab (phase covariant, antisymmetric); t1 = 0.
 * Training: loss = mean |t2 - t2_converged|^2 / 0.05^2 over the unique (a<b, i<j)
 * amplitudes of converged solves, Adam; forward, backward and update are
 * hand-written kernels accumulating in FP32 with BF16-rounded weights and
 * activations (bf16 = 1) or in plain FP32 (bf16 = 0, for gradient checks).  The
 * untrained model (zero output layer) reproduces the MP2 guess exactly.
 * Parameters (exp_mlp_num_params() floats): W1[128][3], b1[128], W2[128][128],
 * b2[128], W3[2][128], b3[2].  Device memory from `alloc`, work on `stream`. */
typedef struct exp_mlp exp_mlp;
int exp_mlp_num_params(void);
exp_status exp_mlp_create(const exp_allocator* alloc, void* stream, uint64_t seed, int bf16, exp_mlp** out);
void exp_mlp_destroy(exp_mlp* mlp);
/* Append the unique amplitudes of every converged instance of ctx as training samples. */
exp_status exp_mlp_add_training_data(exp_mlp* mlp, exp_ctx* ctx);
/* `epochs` passes over the samples in shuffled mini-batches (shuffle seeded by
 * `seed`); loss_out (host, nullable) receives each epoch's mean batch loss. */
exp_status exp_mlp_train(exp_mlp* mlp, int epochs, int batch, double lr, uint64_t seed, double* loss_out);
/* Initial amplitudes of every instance of ctx from the model (replaces the MP2
 * guess; resets DIIS and the iteration count).  Requires exp_init_integrals. */
exp_status exp_mlp_apply(exp_mlp* mlp, exp_ctx* ctx);
/* Copy parameters out (get, host, nullable) and/or in (set, host, nullable). */
exp_status exp_mlp_params(exp_mlp* mlp, float* get, const float* set);
/* Loss and gradient on n host samples: x [n][3] features, tmp2 and target [n][2]
 * (re, im) first-order and target amplitudes; grad (host, num_params). */
exp_status exp_mlp_loss_grad(exp_mlp* mlp, int n, const float* x, const double* tmp2, const double* target,
                             double* loss, float* grad);
/* Samples held, and the mean loss over all of them for the current parameters. */
int64_t exp_mlp_num_samples(const exp_mlp* mlp);
/* Copy samples [first, first+count) to host: x [count][3], tmp2 and target [count][2] (re, im). */
exp_status exp_mlp_samples(exp_mlp* mlp, int64_t first, int64_t count, float* x, float* tmp2, float* target);
exp_status exp_mlp_eval(exp_mlp* mlp, double* loss);
const char* exp_mlp_last_error(const exp_mlp* mlp);

/* Number of kernels this context has launched so far (for launch accounting). */
int64_t exp_kernel_launches(const exp_ctx* ctx);

const char* exp_last_error(const exp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* EXPGB_EXP_H */
