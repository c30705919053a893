/*
 * mwlu.h -- C ABI of the multiword (DD/TD/QD) direct solver and
 * mixed-precision iterative refinement library (libmwlu.so, sm_103a).
 *
 * Method: Kouya, "Accelerated Multiple Precision Direct Method and Mixed
 * Precision Iterative Refinement on Python Programming Environment"
 * (arXiv 2107.12550).  The calls follow the paper's problem statement
 * A x = b (Section 3, Eq. (1)) and the calls of its refinement listing
 * (Section 2, Listing 1): TDLUdecompPM(af, af_ch) -> mw_ludecomp,
 * SolveTDLSPM(xf, af, bf, af_ch) -> mw_solve, the long-precision residual
 * b - a*x -> mw_residual, and the whole loop -> mw_refine.  The paper's
 * multiword block matrix product (BNCmatmul, Section 2) -> mw_gemm_add
 * (C += A B) and mw_gemm_sub (C -= A B), its Strassen form ->
 * mw_gemm_strassen; batches of independent systems -> the *_batched calls.
 *
 * Numbers.  A multiword value of precision w is w binary64 words whose sum
 * is the value: w = 2 double-double (DD), 3 triple-double (TD), 4
 * quad-double (QD); the long precision of the refinement is 8 words
 * (8 x 53 = 424 bits, the paper's 424-bit mpmath precision).
 *
 * Layout (all matrix/vector pointers are DEVICE pointers unless stated):
 *   matrix: w planes of lda*n doubles, column-major, plane = lda*n;
 *           word c of A(i,j) is A[c*lda*n + j*lda + i];  lda >= max(1, n).
 *   vector: w planes of n doubles; word c of v(i) is v[c*n + i].
 *   pivots: int64 (the paper's ctypes c_long array), 0-based, LAPACK swap
 *           sequence: at step k rows k and piv[k] were exchanged.
 * The caller owns every buffer; no call allocates device memory.  Work
 * buffers are caller-provided (size from mw_workspace_size), 256-byte
 * aligned, and must not be shared by calls that may run concurrently.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 * enqueue work and return without synchronising, except mw_refine, which
 * reads a few status words back once per refinement step.  The LU calls
 * (with MW_TUNE_LOOKAHEAD on) fork work onto a second stream the library
 * creates once per device, and join it back into `stream` before
 * returning, so all of a call's work is ordered before anything the caller
 * enqueues on `stream` afterwards (inside a stream capture too: the fork
 * and join become graph edges).  The first such call on a device must run
 * outside a capture; a captured call before it runs the serial schedule.
 * That stream does not survive cudaDeviceReset: after a reset, set
 * MW_TUNE_LOOKAHEAD to 0 or the LU calls return MW_ECUDA.
 *
 * Return codes: MW_OK (0); a negative value -i when argument i (1-based) is
 * invalid; MW_ECUDA when a CUDA call failed (mw_last_cuda_error gives the
 * cudaError_t); MW_ETIMEOUT when a bounded device wait gave up;
 * MW_ESINGULAR / MW_ENOTCONV as documented per call.  Inputs with NaN or
 * Inf give unspecified (but memory-safe) results.  Orders, leading
 * dimensions and GEMM dimensions above 2^28 are rejected as invalid
 * arguments, before any size is computed.
 *
 * Bounded waits.  Kernels whose threads wait for other threads (the
 * substitution's ready values, the panel's candidate records, the split
 * update's copy and MMA barriers, the batched substitution's flags) poll a
 * bounded number of times; a wait that runs out records an error word in
 * the call's work buffer and the kernel returns (its outputs are then
 * incomplete).  The calls that synchronise (mw_refine, the batched
 * refinements) return MW_ETIMEOUT themselves; after an asynchronous call,
 * mw_work_status / mw_batch_work_status / mw_solve_noalloc_status read the
 * error word.
 */
#ifndef MWLU_H
#define MWLU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* precisions: the number of binary64 words */
#define MW_DD 2
#define MW_TD 3
#define MW_QD 4
#define MW_LONG_WORDS 8

/* trailing-update forms of the blocked LU */
#define MW_UPDATE_PLAIN 0 /* multiword GEMM on the FP64 pipe, bitwise equal to unblocked LU */
#define MW_UPDATE_SPLIT 1 /* split-precision (Ozaki-style) tensor-core update (DD only) */

/* status codes */
#define MW_OK 0
#define MW_ESINGULAR 1
#define MW_ENOTCONV 2
#define MW_ECUDA 3
#define MW_ETIMEOUT 4
#define MW_EUNSUPPORTED 5

/* operations for mw_workspace_size */
#define MW_OP_LUDECOMP 0
#define MW_OP_SOLVE 1
#define MW_OP_REFINE 2
#define MW_OP_GEMM 3 /* n = max(m, N) of mw_gemm_sub */

/* stopping tests of mw_refine */
#define MW_STOP_EQ2 0  /* Eq. (2): ||r||_2 <= sqrt(n) rtol ||A||_F ||x||_2 + atol */
#define MW_STOP_BITS 1 /* applied correction <= 2^-(target_bits+2) ||x||_inf */

/*
 * mw_workspace_size -- bytes of work buffer needed by `op` at precision
 * `prec` (for MW_OP_REFINE: the inner precision), trailing-update form
 * `update` and order n.  Writes *bytes (host pointer).  Returns MW_OK or
 * -i for an invalid argument.  Pure host function; no GPU is touched.
 */
int mw_workspace_size(int op, int prec, int update, int64_t n, size_t* bytes);

/*
 * mw_ludecomp -- LU decomposition with partial pivoting in place
 * (Section 2, Listing 1: TDLUdecompPM(af, af_ch)).
 *   prec    MW_DD, MW_TD or MW_QD; the first `prec` planes of A are used.
 *   update  MW_UPDATE_PLAIN (any prec) or MW_UPDATE_SPLIT (MW_DD only).
 *   n       order, n >= 0.
 *   A       device, prec planes (lda, n); overwritten by L\U with the unit
 *           lower factor L implicit.
 *   lda     leading dimension, lda >= max(1, n).
 *   piv     device int64[n]: the swap sequence (0-based).
 *   info    device int64[1]: 0, or k+1 for the first exactly zero pivot
 *           u_kk (the factorisation still completes, as in LAPACK getrf).
 *   work    device work buffer of at least mw_workspace_size(MW_OP_LUDECOMP)
 *           bytes; work_bytes its size.
 * Pivot rule: p = the first row i >= k with the largest |a_ik| under the
 * lexicographic order of the sign-adjusted words (ties take the smallest
 * row).  The plain form is bitwise identical to unblocked right-looking
 * elimination with a rounded multiword multiply and subtraction per element
 * update.  Returns MW_OK, -i, MW_ECUDA or MW_EUNSUPPORTED without waiting
 * for the GPU; a bounded wait that gave up is reported by mw_work_status.
 */
int mw_ludecomp(int prec, int update, int64_t n, double* A, int64_t lda, int64_t* piv,
                int64_t* info, void* work, size_t work_bytes, void* stream);

/*
 * mw_solve -- forward/back substitution with the factors of mw_ludecomp
 * (Section 2, Listing 1: SolveTDLSPM(xf, af, bf, af_ch)).
 *   LU, lda, piv  as produced by mw_ludecomp at precision prec (device).
 *   b             device, prec planes of n (right-hand side).
 *   x             device, prec planes of n (solution); x may equal b.
 * Order of operations per entry: y = P b; y_i -= l_ij y_j for j ascending;
 * d_j = 1 / u_jj (multiword division) for every j, then x_j = y_j * d_j and
 * y_i -= u_ij x_j for j descending.  A zero u_jj gives Inf/NaN entries (check
 * mw_ludecomp's info).  Returns MW_OK, -i or MW_ECUDA without waiting for
 * the GPU; a bounded wait that gave up is reported by mw_work_status.
 */
int mw_solve(int prec, int64_t n, const double* LU, int64_t lda, const int64_t* piv,
             const double* b, double* x, void* work, size_t work_bytes, void* stream);

/*
 * mw_residual -- r = b - A x computed exactly (every product of two words is
 * accumulated in a fixed-point integer covering the whole binary64 product
 * range) and then rounded greedily to r_words words: r_0 = RN(r),
 * r_c = RN(r - r_0 - ... - r_{c-1}).  This is the long-precision residual
 * of Listing 1 (`res = b - a * x`), computed exactly instead of in 424-bit
 * arithmetic.  A: a_words planes (lda, n); b: b_words planes of n; x:
 * x_words planes of n; r: r_words planes of n (all device, 1..8 words).
 * Returns MW_OK, -i or MW_ECUDA.
 */
int mw_residual(int64_t n, const double* A, int64_t lda, int a_words, const double* b,
                int b_words, const double* x, int x_words, double* r, int r_words,
                void* stream);

/*
 * mw_refine -- mixed precision iterative refinement (Section 2, Listing 1).
 *   A, lda, a_words  device matrix (1..8 words; its first `inner` words are
 *                    factored).
 *   b, b_words       device right-hand side (1..8 words).
 *   inner            MW_DD, MW_TD or MW_QD: precision of the LU and solves.
 *   update           trailing-update form for the inner LU.
 *   target_bits      MW_STOP_BITS: stop when the applied correction is below
 *                    2^-(target_bits+2) ||x||_inf.
 *   max_iter         maximum number of corrections (>= 0).
 *   stop_mode        MW_STOP_EQ2 (uses rtol, atol) or MW_STOP_BITS.
 *   x, x_words       device output, x_words planes of n (inner <= x_words
 *                    <= 8; 8 = the paper's 424 bits).
 *   stats            HOST int64[4]: corrections applied, residuals evaluated,
 *                    LU info, final status.
 *   work             device work buffer, mw_workspace_size(MW_OP_REFINE,
 *                    inner, update, n) bytes.
 * Steps: LU of A's first `inner` words; x = solve(b rounded to inner)
 * padded with zero words; loop: r = RN_xw(b - A x) exactly; stop test;
 * e = ilogb(max_i |r_0(i)|); z = solve(first `inner` words of 2^-e r);
 * x = RN_xw(x + 2^e z) exactly.  The MW_STOP_BITS mode also stops (as not
 * converged) when a correction exceeds half the previous one.
 * Returns MW_OK (converged), MW_ESINGULAR (zero pivot; stats[2] = info),
 * MW_ENOTCONV (max_iter reached or stagnation; x holds the last iterate),
 * -i, MW_ECUDA or MW_ETIMEOUT.  Synchronises `stream` once per step.
 */
int mw_refine(int64_t n, const double* A, int64_t lda, int a_words, const double* b,
              int b_words, int inner, int update, int target_bits, int max_iter, int stop_mode,
              double rtol, double atol, double* x, int x_words, int64_t* stats, void* work,
              size_t work_bytes, void* stream);

/*
 * mw_peak_fp64 -- project microbenchmark of the FP64 pipe: runs an
 * independent fused multiply-add stream on every SM and writes the measured
 * rate in FP64 instructions per second to *instr_per_s (host pointer).
 * Synchronous.  Returns MW_OK or MW_ECUDA.
 */
int mw_peak_fp64(double* instr_per_s, void* stream);

/*
 * mw_gemm_sub -- C -= A * B in multiword arithmetic: the block matrix product
 * of the paper's BNCmatmul (Section 2), in the form the blocked LU's
 * trailing update uses.
 *   prec    MW_DD, MW_TD or MW_QD (MW_DD only for MW_UPDATE_SPLIT).
 *   update  MW_UPDATE_PLAIN: each entry applies c -= a_t * b_t for t = 0..K-1
 *           in order with a rounded multiword multiply and subtraction (the
 *           elimination's operation order).  MW_UPDATE_SPLIT: the Ozaki-style
 *           bf16 tensor-core product, per 64-wide slab of K: the slab product is
 *           formed exactly from 15 base-256 digits per operand (pairs of digit
 *           order <= 16), rounded once to DD and subtracted; K must be a
 *           multiple of 64.  Per entry and slab the product error is at most
 *           2^-107 max_t|a_it| max_t|b_tj|.
 *   C       device, prec planes (ldc, N): m x N, updated in place.
 *   A       device, prec planes (lda, K): m x K.   B: prec planes (ldb, N): K x N.
 *   work    device work buffer, mw_workspace_size(MW_OP_GEMM, prec, update,
 *           max(m, N)) bytes.
 * Returns MW_OK, -i, MW_ECUDA or MW_EUNSUPPORTED.
 */
int mw_gemm_sub(int prec, int update, int64_t m, int64_t N, int64_t K, double* C, int64_t ldc,
                const double* A, int64_t lda, const double* B, int64_t ldb, void* work,
                size_t work_bytes, void* stream);

/*
 * mw_gemm_add -- C += A * B: the paper's multiword block matrix product
 * (BNCmatmul, Section 2) as a standalone call; with C zero on entry it is
 * C = A * B.  Arguments, layouts, work buffer and return codes as
 * mw_gemm_sub.
 *   MW_UPDATE_PLAIN: each entry applies c = c + a_t * b_t for t = 0..K-1 in
 *           order (a rounded multiword multiply, then a rounded addition).
 *   MW_UPDATE_SPLIT: per 64-wide slab of K, C + (slab product) formed
 *           exactly and rounded once to DD (the slab product as for
 *           mw_gemm_sub, error at most 2^-107 max_t|a_it| max_t|b_tj| per
 *           entry and slab).
 */
int mw_gemm_add(int prec, int update, int64_t m, int64_t N, int64_t K, double* C, int64_t ldc,
                const double* A, int64_t lda, const double* B, int64_t ldb, void* work,
                size_t work_bytes, void* stream);

/*
 * mw_gemm_strassen -- C = A * B for n x n multiword matrices by Strassen's
 * recursion over the block matrix product (the paper's Strassen form of
 * BNCmatmul, Section 2): `levels` levels of seven half-size products and 18
 * rounded multiword additions (Strassen 1969; the order of the additions is
 * listed in strassen.cu), then the block product from a zero C
 * (mw_gemm_add's plain or split form) on blocks of n / 2^levels.
 *   prec, update  as mw_gemm_add (split: MW_DD and (n >> levels) % 64 == 0).
 *   levels  0..8; n must be divisible by 2^levels (else MW_EUNSUPPORTED).
 *           levels = 0 is mw_gemm_add from a zero C.
 *   A, B    device, prec planes (lda, n) / (ldb, n): n x n, not overwritten.
 *   C       device, prec planes (ldc, n): overwritten with A * B; must not
 *           overlap A or B.
 *   work    mw_gemm_strassen_workspace_size(...) bytes (the temporaries:
 *           9 (n/2^l)^2 prec doubles per level l, and the split scratch).
 * The result differs from the classical product by roundings: the error
 * bound grows by about a factor 12 per level instead of 2 (Higham, Accuracy
 * and Stability of Numerical Algorithms, Section 23.2.2).
 * Returns MW_OK, -i, MW_EUNSUPPORTED or MW_ECUDA.
 */
int mw_gemm_strassen_workspace_size(int prec, int update, int levels, int64_t n, size_t* bytes);
int mw_gemm_strassen(int prec, int update, int levels, int64_t n, const double* A, int64_t lda,
                     const double* B, int64_t ldb, double* C, int64_t ldc, void* work, size_t work_bytes,
                     void* stream);

/*
 * Batches of independent systems of uneven order (one launch per step for
 * the whole batch: the batched persistent form of the method).
 *   count    number of systems; n_host: HOST int32[count], 1 <= n[s] <= 1024.
 *   Layout (device): with moff[s] = sum_{s'<s} n[s']^2 and
 *   voff[s] = sum_{s'<s} n[s'], system s's matrix of w words is at
 *   M + w*moff[s] (word c of M_s(i,j) at M[w*moff[s] + c*n*n + j*n + i],
 *   column-major, ld = n); a vector of w words at v + w*voff[s] (word c of
 *   v_s(i) at v[w*voff[s] + c*n + i]); pivots at piv + voff[s]; info[s].
 *   The library derives the offsets and a largest-first processing order
 *   from n_host and uploads them into the work buffer on every call.
 * Each system's results are bitwise identical to the single-system calls
 * (mw_ludecomp/mw_solve/mw_refine with MW_UPDATE_PLAIN, MW_STOP_BITS).
 * The persistent kernels give each system to one CTA, taken from an atomic
 * counter: no CTA waits for another.
 */
int mw_batch_workspace_size(int op, int prec, int count, const int* n_host, size_t* bytes);
int mw_ludecomp_batched(int prec, int count, const int* n_host, double* A, int64_t* piv, int64_t* info,
                        void* work, size_t work_bytes, void* stream);
int mw_solve_batched(int prec, int count, const int* n_host, const double* LU, const int64_t* piv,
                     const double* b, double* x, void* work, size_t work_bytes, void* stream);
/* stats: DEVICE int64[4*count]: corrections, residuals, LU info, status
 * (MW_OK, MW_ENOTCONV, MW_ESINGULAR, or MW_ETIMEOUT when a bounded wait
 * gave up) per system.  x: x_words planes per system (inner <= x_words <=
 * 8).  Reads one int back per refinement step, except inside a stream
 * capture (see mw_batch_plan_cache). */
int mw_refine_batched(int count, const int* n_host, const double* A, int a_words, const double* b,
                      int b_words, int inner, int target_bits, int max_iter, double* x, int x_words,
                      int64_t* stats, void* work, size_t work_bytes, void* stream);

/*
 * Blocked batched LU (Section 2: the blocked LU with its block matrix
 * product, applied to a whole batch at once).  Same packed layout, pivots,
 * info and stats as above; n[s] <= 1024.  All systems advance one panel of
 * 64 columns per step: the panels of the systems still active (one CTA
 * each), their row swaps and U12 = L11^-1 A12, then ONE trailing-update
 * launch over the tiles of every active system.
 *   update   MW_UPDATE_PLAIN: the plain multiword GEMM; every system's
 *            factors are bitwise identical to mw_ludecomp / the persistent
 *            mw_ludecomp_batched.
 *            MW_UPDATE_SPLIT (DD only, else MW_EUNSUPPORTED): the
 *            split-precision tensor-core GEMM of mw_ludecomp, with its
 *            per-entry error bound 2^-107 max|l| max|u| per update.
 * mw_batch_blocked_workspace_size: op MW_OP_LUDECOMP or MW_OP_REFINE; the
 *   work buffer holds the plan, the per-step tile lists and, for the split
 *   update, the bf16 digit slices of the largest step.
 * mw_refine_batched_blocked: mw_refine_batched with the inner LU factored by
 *   the blocked batched LU (`update` as above; split needs inner = MW_DD).
 * Returns MW_OK, -i, MW_ECUDA or MW_EUNSUPPORTED.
 */
int mw_batch_blocked_workspace_size(int op, int prec, int update, int count, const int* n_host,
                                    size_t* bytes);
int mw_ludecomp_batched_blocked(int prec, int update, int count, const int* n_host, double* A,
                                int64_t* piv, int64_t* info, void* work, size_t work_bytes, void* stream);
int mw_refine_batched_blocked(int count, const int* n_host, const double* A, int a_words,
                              const double* b, int b_words, int inner, int update, int target_bits,
                              int max_iter, double* x, int x_words, int64_t* stats, void* work,
                              size_t work_bytes, void* stream);

/*
 * Resident batch plans, for CUDA graph capture of the batched calls.
 * Every batched call uploads its plan (offsets, processing order, tile
 * lists) into the work buffer with host-to-device copies, which a stream
 * capture cannot record from pageable memory.  mw_batch_plan_cache(1)
 * switches on a host-side record of the plans already resident per work
 * buffer address: a call whose plan (same kind, batch, precision and update)
 * is already in its work buffer then issues no copy, so after one ordinary
 * call the same calls on the same buffers can be captured and replayed.
 * The caller must keep those work buffers alive and unmodified while the
 * record is on (a freed buffer's address can come back holding other data).
 *   mw_batch_plan_cache(on)  returns the previous setting; off forgets all.
 *   mw_batch_plan_reset()    forgets all records.
 * The batched refinements can be captured too: called while their stream
 * is being captured, they record the refinement loop as a graph while node
 * (CUDA conditional node) whose condition a kernel sets at the end of each
 * step to "systems still running", so a replay reads nothing back; outside
 * a capture they read one integer per step instead.  The first call on a
 * device must run outside a capture (it also creates the library's stream
 * into which the loop body is captured).  Per-system results, including
 * MW_ETIMEOUT, are in `stats`.
 */
int mw_batch_plan_cache(int on);
int mw_batch_plan_reset(void);

/*
 * mw_arith -- element-wise multiword arithmetic on device arrays (the
 * DD/TD/QD building blocks of Section 1, as used inside every kernel):
 *   op 0: z = x + y   1: z = x - y   2: z = x * y   3: z = x / y
 *   op 4: z plane 0 = sign(|x| - |y|) in the pivot order (-1, 0, +1),
 *         other planes 0.
 * x, y, z: device, prec planes of cnt doubles, 0 <= cnt <= 256 (2^31 - 1)
 * (-3 otherwise, on the host).  Asynchronous on `stream`.
 * Returns MW_OK, -i or MW_ECUDA.
 */
int mw_arith(int op, int prec, int64_t cnt, const double* x, const double* y, double* z,
             void* stream);

/*
 * Launch accounting and per-phase timing.  Phases: 0 panel factorisation,
 * 1 row interchanges, 2 triangular solve of U12, 3 plain trailing update,
 * 4 split trailing update (tensor-core GEMMs), 5 substitution, 6 pivot
 * permutation, 7 exact residual, 8 refinement bookkeeping, 9 split-update
 * slicing, 10 batched persistent LU, 11 batched substitution, 12 the inner
 * tensor-core products of the split LU's recursive panel.
 * mw_profile_enable(1) brackets every later kernel launch of the library with
 * two CUDA events on its stream (0 turns this off; launches are counted
 * either way).  mw_profile_read synchronises on the recorded events and
 * writes, for phases 0..nphase-1, the summed device time in ms (ms, host
 * array, may be NULL) and the launch count (launches, host array, may be
 * NULL); reset != 0 clears both afterwards.  Returns MW_OK or MW_ECUDA.
 */
int mw_profile_enable(int on);
int mw_profile_read(double* ms, long long* launches, int nphase, int reset);

/*
 * mw_solve_noalloc -- the substitution of mw_solve for callers that cannot
 * allocate device memory and so cannot pass a work buffer: code inside a
 * framework whose memory pool owns the whole GPU and forbids outside
 * allocations, plugins or hooks that are not allowed to allocate, and
 * latency-critical loops that must stay away from the allocator.  The paper
 * has no counterpart; this is an interface convenience of this library.
 *   Arguments and results are those of mw_solve without work/work_bytes:
 *   the caller still passes LU, lda, piv, b and x (device pointers).
 *   Scratch: a fixed array of MW_NOALLOC_SCRATCH_BYTES in the library's own
 *   device memory, held on every GPU that loads the library until exit.  n
 *   is limited to the orders whose scratch fits (mw_workspace_size(
 *   MW_OP_SOLVE, prec, 0, n) <= MW_NOALLOC_SCRATCH_BYTES: n <= 20968 for QD,
 *   27584 for TD, 40320 for DD); larger n returns -2 before any GPU work.
 *   Nothing is allocated or freed by this call.
 *   Set-up: the first call on each device looks up the scratch address with
 *   cudaGetSymbolAddress (with that device current) and caches it; make that
 *   first call outside any stream capture.  The cache does not survive
 *   cudaDeviceReset: after a reset the library's device memory is loaded
 *   again at another address, so do not call this entry point after
 *   resetting a device it has been used on.
 *   Orders above 40320 (the largest that fits at any precision) are
 *   rejected before any size is computed.
 *   Error word: a bounded wait that gave up is recorded in the scratch;
 *   mw_solve_noalloc_status reads it.
 *   Sharing: all calls on a device use the same scratch, which keeps the last
 *   call's contents (the parts that must start at zero are cleared by each
 *   call); calls that overlap on the GPU, e.g. on two streams at once, race
 *   on it and must be serialised by the caller.
 * Returns MW_OK, -i or MW_ECUDA.
 */
#define MW_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u)
int mw_solve_noalloc(int prec, int64_t n, const double* LU, int64_t lda, const int64_t* piv,
                     const double* b, double* x, void* stream);

/*
 * Tuning knobs (process-wide, per precision; read at each launch).  They
 * change the blocking only: every plain-path result is bitwise the same for
 * any value (the split path's leaf widths change roundings only).
 *   MW_TUNE_PANEL_WIDTH          panel width nb of the plain blocked LU:
 *                                32, 64 (default) or 128 (the split update
 *                                always uses 64)
 *   MW_TUNE_PANEL_ROWS_PER_CTA   panel rows per CTA before the panel kernel
 *                                adds CTAs: 1..4096 (default 8)
 *   MW_TUNE_SPLIT_PANEL_LEAF     the split (DD) LU of one system factors each
 *                                64-column panel recursively down to leaves of
 *                                this width (8, 16 or 32), the inner updates
 *                                as split products; 0: no recursion below 64
 *                                (the default, chosen by measurement; the
 *                                results differ by roundings only).
 *   MW_TUNE_BATCH_CTAS_PER_SM    persistent CTAs per SM of the batched LU:
 *                                1..8 (default 2)
 *   MW_TUNE_GEMM_TILE            tile of the plain trailing update of one
 *                                system (and of mw_gemm_sub): 0 (default)
 *                                picks per launch the tile with the least
 *                                per-SM work, ceil(tiles / SMs) x tile size,
 *                                the smaller on a tie (all three run a full
 *                                wave at the same rate); 1, 2, 3 force the
 *                                large, middle or small tile (DD 64x64,
 *                                32x64, 32x32; TD 32x64, 16x32, 16x16; QD
 *                                32x32, 16x32, 16x16, rows x columns)
 *   MW_TUNE_BATCH_SPLIT_LEAF     the blocked batched split (DD) LU factors
 *                                each 64-column panel recursively down to
 *                                leaves of this width (8, 16 or 32; default
 *                                8), the wider inner updates as split
 *                                products; the results differ by roundings
 *                                only, within the split path's error bound
 *   MW_TUNE_LOOKAHEAD            1 (default): mw_ludecomp (and the LU inside
 *                                mw_refine) updates the next panel's columns
 *                                first and factors that panel on a second,
 *                                higher-priority stream while the rest of
 *                                the trailing matrix is updated; 0: one
 *                                stream, panel after update.  Every entry
 *                                receives the same operations in the same
 *                                order either way: bitwise the same result.
 * mw_set_tuning returns the previous value, or -1 (param), -2 (prec) or
 * -3 (value) when invalid; mw_get_tuning returns the value or -1/-2.
 */
#define MW_TUNE_PANEL_WIDTH 0
#define MW_TUNE_PANEL_ROWS_PER_CTA 1
#define MW_TUNE_BATCH_CTAS_PER_SM 2
#define MW_TUNE_SPLIT_PANEL_LEAF 3
#define MW_TUNE_GEMM_TILE 4
#define MW_TUNE_BATCH_SPLIT_LEAF 5
#define MW_TUNE_LOOKAHEAD 6
int mw_set_tuning(int param, int prec, int value);
int mw_get_tuning(int param, int prec);

/*
 * mw_work_status -- synchronises `stream`, then reports whether a bounded
 * device wait gave up in the last call that used the single-system work
 * buffer `work` for operation `op` (MW_OP_LUDECOMP, MW_OP_SOLVE or
 * MW_OP_GEMM) with trailing-update form `update`: MW_OK, MW_ETIMEOUT, -i or
 * MW_ECUDA.  Every such call clears the error word when it starts.
 *
 * mw_batch_work_status -- the same for the work buffer of any batched call
 * (mw_*_batched, mw_*_batched_blocked): the error word sits in the buffer's
 * head and is cleared at the start of every batched call.
 *
 * mw_solve_noalloc_status -- the same for the fixed scratch of
 * mw_solve_noalloc on the current device.
 */
int mw_work_status(int op, int update, const void* work, void* stream);
int mw_batch_work_status(const void* work, void* stream);
int mw_solve_noalloc_status(void* stream);

/*
 * mw_set_wait_limit -- the number of polls after which the bounded waits of
 * the substitution, the panel factorisation and the batched substitution
 * give up, for every later launch in the process (0, the default: each
 * kernel's own limit, which corresponds to seconds of waiting).  A small
 * value makes those waits run out on purpose, to exercise the error path
 * (the kernels return and the status calls report MW_ETIMEOUT; nothing
 * hangs or faults).  Returns the previous value, or -1 for polls < 0.
 */
long long mw_set_wait_limit(long long polls);

/* mw_strerror -- static text for a status code. */
const char* mw_strerror(int code);

/* mw_last_cuda_error -- the cudaError_t behind the last MW_ECUDA. */
int mw_last_cuda_error(void);

/* mw_version -- library version string. */
const char* mw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MWLU_H */
