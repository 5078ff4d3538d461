/*
 * cqr.h - C ABI of the GB300 (sm_103a) FP64 CholeskyQR library.
 *
 * QR factorisation A = Q R of tall-and-skinny FP64 matrices (m >= n) by the
 * modified CholeskyQR2 with block Gram-Schmidt (mCQR2GS, arXiv 2405.04237,
 * Sec. 5.4, Alg. 9), CholeskyQR2 with Gram-Schmidt (CQR2GS, Sec. 5.3, Alg. 6
 * and Alg. 7), CholeskyQR2 (Sec. 4, Alg. 3) and shifted CholeskyQR3 (Sec. 5.2,
 * Alg. 4 and Alg. 5), plus the reverse-mode adjoint of A = Q R.
 *
 * Conventions shared by every entry point
 *   - All matrices are FP64, column-major, with leading dimension >= rows.
 *   - Matrix and workspace pointers are DEVICE pointers owned by the caller
 *     (except where an argument says "host").  The library never allocates
 *     device memory itself: the caller passes a workspace of at least the
 *     size the matching *_workspace_size() function returns, 256-byte
 *     aligned, or passes workspace = NULL to have it taken from an allocator
 *     the caller registered with cqr_set_allocator() (see there).
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and returns without synchronising.  Every launch is
 *     asynchronous and graph-capturable: no allocation, no host sync.
 *   - The return value reports argument errors only, LAPACK style: 0 = ok,
 *     -i = argument i (1-based) invalid; CQR_ERR_CUDA if a launch failed.
 *     Numerical failure (a Cholesky breakdown: the Gram matrix is not
 *     numerically positive definite, Sec. 3) is reported through a device
 *     status word kept at the start of the workspace; read it with
 *     cqr_read_status() (synchronous) after the stream work completes.
 *     Status codes: 0 = ok; j+1 (> 0) = breakdown at global column j of the
 *     factorisation; CQR_STATUS_TIMEOUT = a bounded wait inside a kernel
 *     (an mbarrier of the emulated products, bounded at 2 s) expired.  After
 *     a breakdown or a timeout, every later kernel of the same call returns
 *     immediately and Q, R are undefined.
 */
#ifndef CQR_GB300_H
#define CQR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cqr_stream_t; /* identical to cudaStream_t */

enum cqr_variant {
  CQR_MCQR2GS = 0, /* Alg. 9: CQR2 on panel 1, then per panel: project, CQR, re-orthogonalise, CQR */
  CQR_CQR2GS = 1,  /* Alg. 7: CQRGS (Alg. 6) twice, R = R2 R1 */
  CQR_CQR2 = 2,    /* Alg. 3: CholeskyQR twice on the whole matrix (panel_b ignored, b = n) */
  CQR_SCQR3 = 3    /* Alg. 5: shifted CholeskyQR (Alg. 4) then CholeskyQR2, R = R2 R1 (b = n) */
};

/* Flag OR-ed into `variant` of cqr_factor (MCQR2GS, CQR2GS): look-ahead, the
 * overlap of each trailing update with the next panel's CholeskyQR that
 * Sec. 7 names as future work.  The update of step j is split: the next
 * panel's columns on `stream`, the rest concurrently on a library-owned side
 * stream joined back with an event before the next projection.  Results are
 * bitwise identical to the default schedule.  Off by default: on GB300 the
 * path is bound by the FP64 pipe with almost no idle gaps, so the overlap
 * measured no gain (20,000 x 64 to 2^21 x 1024). */
#define CQR_LOOKAHEAD 0x100

/* Flag OR-ed into `variant` of cqr_factor (MCQR2GS only; other variants give
 * argument error -10): the runtime choice of how many CholeskyQR passes a
 * panel gets, the optimisation Sec. 7 proposes.  For the second pass of each
 * panel (Alg. 3 step 2 on panel 1, Alg. 9 step 8 on the others), if every
 * entry of its Cholesky factor S2 lies within 8u of the identity (u = 2^-53),
 * the panel is already orthonormal to working precision: S2 := I exactly
 * and the triangular solve is skipped (decided on the device, no host
 * synchronisation).  Only nearly orthonormal panels qualify: on the paper's
 * test matrices the rule fires for kappa ~ 1 and never for kappa >= 1e2. */
#define CQR_ADAPTIVE 0x200

/* Flag OR-ed into `variant` of cqr_factor and cqr_workspace_size (MCQR2GS
 * only): every m-row product of Alg. 9 -- the Gram matrices W = X^T X
 * (Alg. 1 step 1), the projections Y = Q_{j-1}^T A_{j:k} and
 * Z = Q_{1:j-1}^T P (steps 3 and 7) and the updates A_{j:k} -= Q_{j-1} Y
 * and P -= Q_{1:j-1} Z (steps 4 and 7) -- runs on the FP8 tensor cores
 * (tcgen05, accumulators in TMEM) with an error-free splitting of the FP64
 * operands (Ozaki scheme): each operand is scaled by powers of two along
 * the contraction (per column and 4096-row sub-chunk for a Gram matrix or
 * projection, per row for an update) and cut into 14 signed 4-bit digits
 * (56 bits); the 105 most significant digit-plane pairs are multiplied
 * exactly (FP32 accumulation of integers < 2^24) and recombined with one
 * rounding.  Not FP64 arithmetic, but FP64-accurate: the truncation drops
 * terms below about 2^-52 of the scales' product.  The Cholesky
 * factorisations and the substitutions of the triangular solves stay native
 * FP64; a solve runs in 32-column substitution blocks, and the products that
 * couple the blocks (X_2 -= X_1 U_12, m rows) are emulated like the other
 * m-row products.  The update runs
 * unsplit on the caller's stream, so CQR_LOOKAHEAD has no effect with this
 * flag.  The workspace grows (cqr_workspace_size with the flag) by the digit
 * planes of one row chunk (1 to 2 GiB) and one FP64 partial per 4096 rows. */
#define CQR_EMULATED 0x400

/* Flag OR-ed into `variant` of cqr_factor and cqr_workspace_size (MCQR2GS
 * only; not with CQR_EMULATED or CQR_LOOKAHEAD): adaptive panel width, the
 * paper's remedy for a Cholesky breakdown -- a smaller b lowers every
 * panel's condition number (Sec. 5.3-5.4, Eq. cond_bounds).  The first
 * CholeskyQR of each panel (Alg. 9 step 1's first pass, step 6) is tested:
 * the panel is rejected when its Cholesky factorisation breaks down or
 * (max U_ii / min U_ii)^2 > 1/(64 u), u = 2^-53 (its Gram matrix within a
 * factor 64 of numerical singularity).  A rejected panel is left untouched
 * and retried with the largest divisor of b that is <= b/2; every later
 * panel keeps the new width.  A one-column panel is never rejected (its
 * breakdown is reported as usual).  With no rejection the result is bitwise
 * that of the fixed width.  The decision is read on the host before each
 * triangular solve, so the call SYNCHRONISES `stream` once per panel
 * attempt and cannot be captured into a CUDA graph.  The final width is
 * left in the workspace; read it with cqr_read_panel_width(). */
#define CQR_HALVE 0x800

#define CQR_ERR_CUDA (-1000)
#define CQR_STATUS_TIMEOUT (-2000)
#define CQR_ERR_NOALLOC_TOO_LARGE (-3000)
#define CQR_ERR_ALLOC (-4000)

/*
 * Caller-registered allocator for calls made with workspace = NULL.
 *   cqr_alloc_fn(bytes, stream, ctx) returns DEVICE memory of at least
 *     `bytes`, 256-byte aligned, usable on `stream` (NULL = failure);
 *   cqr_free_fn(ptr, bytes, stream, ctx) takes it back.
 * A call with workspace = NULL (cqr_factor, cqr_factor_host, cqr_backward,
 * cqr_factor_batched) asks for exactly the *_workspace_size() bytes,
 * enqueues its work, SYNCHRONISES `stream`, then frees the memory -- so any
 * allocator works (cudaMalloc/cudaFree, a caching allocator, a pool), and
 * the call is synchronous and cannot be captured into a CUDA graph.
 * cqr_factor then returns the status word itself (0, breakdown column + 1,
 * or CQR_STATUS_TIMEOUT) instead of leaving it in the workspace.  Without a
 * registered allocator workspace = NULL is an argument error; an allocation
 * that fails or is misaligned returns CQR_ERR_ALLOC.
 */
typedef void* (*cqr_alloc_fn)(size_t bytes, struct CUstream_st* stream, void* ctx);
typedef void (*cqr_free_fn)(void* ptr, size_t bytes, struct CUstream_st* stream, void* ctx);

/*
 * cqr_set_allocator: registers (alloc, free, ctx) for every later
 * workspace = NULL call of this process; (NULL, NULL) unregisters.
 * Returns 0, -1 (free without alloc) or -2 (alloc without free).
 */
int cqr_set_allocator(cqr_alloc_fn alloc, cqr_free_fn free_fn, void* ctx);

/* Largest panel width the library accepts (the one-CTA Cholesky keeps a
 * b x b Gram matrix in shared memory up to 128 and in L2 above).  CQR_CQR2
 * and CQR_SCQR3 factor the whole matrix as one panel (b = n), so they
 * accept n <= CQR_MAX_PANEL only (argument error -2 beyond). */
#define CQR_MAX_PANEL 512

/*
 * cqr_workspace_size: bytes of device workspace cqr_factor() needs for an
 * m x n factorisation with panel width panel_b (0 = library default, see
 * cqr_default_panel) and the given variant (with its CQR_EMULATED flag, if
 * any).  Returns 0 for invalid sizes.
 */
size_t cqr_workspace_size(int64_t m, int64_t n, int panel_b, int variant);

/*
 * cqr_default_panel: the panel width used when panel_b == 0: the largest
 * divisor of n that is <= min(256, ceil(n/3)), i.e. at least three panels,
 * the count the paper found stable for condition numbers up to 1e15
 * (Sec. 5.4, Fig. 6), and a divisor so that k = n/b is an integer (Alg. 6).
 */
int cqr_default_panel(int64_t n);

/*
 * cqr_factor: A = Q R.
 *   m, n       rows and columns, m >= n >= 1; n <= CQR_MAX_PANEL for
 *              CQR_CQR2 and CQR_SCQR3                              (args 1, 2)
 *   A, lda     input, m x n, lda >= m.  Read-only unless Q == A    (args 3, 4)
 *   panel_b    panel width b; must divide n; 0 = cqr_default_panel(n).
 *              Ignored by CQR_CQR2 and CQR_SCQR3 (b = n)            (arg 5)
 *   Q, ldq     output m x n with orthonormal columns, ldq >= m.  Q may be
 *              A itself (in-place factorisation, ldq == lda); otherwise Q
 *              must not overlap A                                   (args 6, 7)
 *   R, ldr     output n x n upper triangular with positive diagonal;
 *              its strict lower triangle is zeroed; ldr >= n        (args 8, 9)
 *   variant    enum cqr_variant, optionally | CQR_LOOKAHEAD, CQR_ADAPTIVE,
 *              CQR_EMULATED, CQR_HALVE                               (arg 10)
 *   workspace  device buffer of ws_bytes >= cqr_workspace_size(), or
 *              NULL: taken from the registered allocator, the call
 *              synchronises and returns the status word (see
 *              cqr_set_allocator)                                  (args 11, 12)
 *   stream     CUDA stream                                          (arg 13)
 * Panel loop (Alg. 9): for each panel j the Gram W_j = A_j^T A_j (Alg. 1
 * step 1), the b x b Cholesky W_j = U^T U (step 2), the triangular solve
 * Q_j = A_j U^{-1} (step 3), the projection Y = Q_{j-1}^T A_{j:k} and the
 * update A_{j:k} -= Q_{j-1} Y (Alg. 9 steps 3-4), and the interleaved
 * CQR / re-orthogonalisation / CQR of the panel (Alg. 9 steps 6-8), with
 * R_jj = S2 S1 and R_{1:j-1,j} += Z S1.
 */
int cqr_factor(int64_t m, int64_t n, double* A, int64_t lda, int panel_b, double* Q, int64_t ldq, double* R,
               int64_t ldr, int variant, void* workspace, size_t ws_bytes, cqr_stream_t stream);

/*
 * cqr_factor_noalloc: cqr_factor() for callers that cannot allocate device
 * memory when they factor -- code working inside a memory budget fixed at
 * start-up, code called back from within another framework's allocator or
 * memory pool, code with a no-allocation-after-initialisation rule.  The
 * paper has no counterpart; this is a library convenience.
 *   Arguments 1-9 as in cqr_factor.  Argument 10 is a plain variant (enum
 *   cqr_variant) without flags: CQR_LOOKAHEAD, CQR_ADAPTIVE and CQR_EMULATED
 *   are refused with -10.  There is no workspace argument: the scratch is a
 *   file-scope device array of CQR_NOALLOC_SCRATCH_BYTES (64 MiB) that every
 *   GPU which loads the library holds until the process exits.  Under the
 *   CUDA runtime's lazy module loading (the default) the array is created on
 *   a device by the first cqr_factor_noalloc call there, so make that first
 *   call during initialisation.
 *   status   DEVICE int*: receives the status word (0, breakdown column + 1)
 *            when the stream reaches the end of the call; NULL = not reported
 *            (arg 11)
 *   stream   CUDA stream (arg 12)
 * Returns the same argument codes as cqr_factor, or
 * CQR_ERR_NOALLOC_TOO_LARGE when the sizes need more scratch than the array
 * holds (compare cqr_workspace_size() with CQR_NOALLOC_SCRATCH_BYTES); nothing
 * is launched then.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls share the one array and it keeps
 * the last call's contents (each call clears what must start at zero), so
 * calls whose work overlaps on the GPU -- on different streams, or from
 * different threads -- race and give wrong results; order them on one stream
 * or synchronise between them.  The results are the same as cqr_factor()'s.
 */
#define CQR_NOALLOC_SCRATCH_BYTES (64ull << 20)
int cqr_factor_noalloc(int64_t m, int64_t n, double* A, int64_t lda, int panel_b, double* Q, int64_t ldq, double* R,
                       int64_t ldr, int variant, int* status, cqr_stream_t stream);

/*
 * cqr_factor_host: A = Q R with A, Q and R in HOST memory; the library moves
 * them to and from the caller's device buffers and overlaps those copies with
 * the factorisation.  The paper times factorisations of resident matrices;
 * this is the call for a matrix that lives in host memory.
 *   Arguments 1-10 as in cqr_factor, but A, Q and R are host pointers
 *   (column-major, leading dimensions lda, ldq, ldr).  Q may be A itself
 *   (ldq == lda); otherwise the two must not overlap (-6).
 *   Qd, ldqd   DEVICE buffer, m x n, ldqd >= m: receives A, is factored in
 *              place and holds Q on return                          (args 11, 12)
 *   Rd, ldrd   DEVICE buffer, n x n, ldrd >= n: holds R on return; must not
 *              overlap Qd                                            (args 13, 14)
 *   workspace, ws_bytes, stream  as in cqr_factor, sized by the same
 *              cqr_workspace_size(m, n, panel_b, variant)          (args 15-17)
 * Schedule for CQR_MCQR2GS (Alg. 9), on `stream` and one library-owned copy
 * stream per device: the first panel's b columns are copied in first and its
 * CholeskyQR2 (step 1) starts as soon as they have arrived, while the other
 * n - b columns are copied in behind it; the first projection (steps 3-5)
 * waits for them.  Each panel Q_j is final after its second CholeskyQR
 * (step 8) and is never written again, so it is copied out at once, while
 * later panels compute; R is copied out at the end.  Only the first panel's
 * copy in and the last panel's copy out are not hidden.  The other variants
 * copy A in, factor and copy Q and R out, in that order.  The kernels and
 * their order are those of cqr_factor with the same arguments, so Qd, Rd and
 * the host results are bitwise cqr_factor's.  Page-locked host buffers
 * (cudaHostAlloc, cudaHostRegister) are needed for the overlap; pageable ones
 * give the same results, but the CUDA runtime then makes the copies
 * synchronous, so the host waits for each one.
 * Returns the argument codes of cqr_factor (-3: A == NULL; -6: Q == NULL or
 * overlapping A; -8: R == NULL), -13 (Qd == NULL), -14 (ldqd < m), -15
 * (Rd == NULL or overlapping Qd), -16 (ldrd < n), or CQR_ERR_CUDA.  Like
 * cqr_factor it returns once the work is enqueued (the host results are
 * complete when `stream` is); with CQR_HALVE, or with workspace == NULL, it
 * synchronises `stream` first.  The status word is left in the workspace
 * (cqr_read_status), or returned for workspace == NULL.
 */
int cqr_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int panel_b, double* Q, int64_t ldq,
                    double* R, int64_t ldr, int variant, double* Qd, int64_t ldqd, double* Rd, int64_t ldrd,
                    void* workspace, size_t ws_bytes, cqr_stream_t stream);

/*
 * cqr_read_panel_width: synchronises `stream`, then copies into *panel_b
 * (host) the width of the last panel of the last CQR_HALVE call that used
 * `workspace` (not written by calls without the flag, nor when the
 * workspace was NULL).  Returns 0, -1 for a NULL argument, or CQR_ERR_CUDA.
 */
int cqr_read_panel_width(const void* workspace, cqr_stream_t stream, int* panel_b);

/*
 * cqr_read_status: synchronises `stream`, then copies the status word of the
 * last call that used `workspace` into *status (host).  Returns 0, or
 * CQR_ERR_CUDA if the copy failed.
 */
int cqr_read_status(const void* workspace, cqr_stream_t stream, int* status);

/*
 * cqr_backward_workspace_size: device workspace bytes cqr_backward() needs.
 */
size_t cqr_backward_workspace_size(int64_t m, int64_t n);

/*
 * cqr_backward: reverse-mode adjoint of A = Q R (not in the paper; the
 * standard QR rule):  M = R Rbar^T - Qbar^T Q;  B = Qbar + Q copyltu(M),
 * copyltu(M) = tril(M) + tril(M,-1)^T;  Abar = B R^{-T} (row-wise
 * substitution against R^T).
 *   m, n       sizes, m >= n >= 1                                   (args 1, 2)
 *   Q, ldq     forward output Q (m x n)                             (args 3, 4)
 *   R, ldr     forward output R (n x n upper, nonsingular)          (args 5, 6)
 *   dQ, lddq   upstream gradient Qbar (m x n); NULL means zero      (args 7, 8)
 *   dR, lddr   upstream gradient Rbar (n x n); NULL means zero;
 *              only its upper triangle influences the result        (args 9, 10)
 *   dA, ldda   output Abar (m x n); must not overlap the inputs     (args 11, 12)
 *   workspace, ws_bytes, stream  as in cqr_factor (NULL workspace:
 *              registered allocator, synchronous, returns 0)      (args 13-15)
 * Uses the same Gram/projection, update and triangular-solve kernels as the
 * forward pass.  The status word is not used (R is assumed nonsingular).
 */
int cqr_backward(int64_t m, int64_t n, const double* Q, int64_t ldq, const double* R, int64_t ldr,
                 const double* dQ, int64_t lddq, const double* dR, int64_t lddr, double* dA, int64_t ldda,
                 void* workspace, size_t ws_bytes, cqr_stream_t stream);

/*
 * cqr_batched_workspace_size: device workspace bytes for a batch, given the
 * HOST arrays of sizes and panel widths (panel_b[i] == 0 = default).
 */
size_t cqr_batched_workspace_size(int batch, const int64_t* m, const int64_t* n, const int* panel_b, int variant);

/* Flags OR-ed into `variant` of cqr_factor_batched and
 * cqr_batched_workspace_size.  CQR_BATCH_POOL forces the stream-pool
 * schedule; CQR_BATCH_GROUP(G) sets the CTAs per matrix of the persistent
 * launch (G must divide the SM count; 0 = default, the largest divisor
 * <= 8); CQR_HALVE (persistent path only) applies the adaptive panel width
 * on the device. */
#define CQR_BATCH_POOL 0x1000
#define CQR_BATCH_GROUP(G) ((G) << 16)

/*
 * cqr_factor_batched: factors `batch` independent matrices A_i = Q_i R_i
 * (variant CQR_MCQR2GS or CQR_CQR2GS).  Not in the paper (batching of many
 * small problems); each matrix follows Alg. 9 / Alg. 7 as cqr_factor()
 * does.  Two schedules:
 *   persistent (mCQR2GS, every n_i <= 128, n_i and b_i multiples of 4,
 *   unless CQR_BATCH_POOL): ONE cooperative kernel launch with one CTA per
 *   SM.  Groups of G CTAs take whole matrices (a static largest-first
 *   schedule); the G CTAs of a group split the matrix's rows (the row-block
 *   distribution of Alg. 2 / Alg. 8), write partial sums of every m-row
 *   product to their own slots, meet at a group barrier and add the slots
 *   in rank order, each factoring the b x b Gram matrix redundantly (the
 *   redundant Cholesky of Alg. 2).  Each pass over a sub-block of rows
 *   fuses a streaming step with the next m-row product (update + Gram,
 *   solve + projection, re-orthogonalisation + Gram).  Results match the
 *   single-matrix path to rounding (a different summation order), not
 *   bitwise.  Every group-barrier wait is bounded (2 s); on expiry the
 *   unfinished matrices get CQR_STATUS_TIMEOUT.  With CQR_HALVE a rejected
 *   panel (see CQR_HALVE) is retried at half width on the device; read the
 *   final widths with cqr_batched_panel_widths().
 *   stream pool (CQR2GS, wider matrices, or CQR_BATCH_POOL): each matrix
 *   runs exactly the kernel sequence of a cqr_factor() call with the same
 *   sizes and panel width (so its result is bitwise that call's), the
 *   matrices spread over library-owned streams forked from and joined back
 *   into `stream`.
 *   batch                  number of matrices, >= 0                  (arg 1)
 *   m, n, lda, panel_b     HOST arrays of length batch                (args 2-5)
 *   A, Q, R                HOST arrays of DEVICE pointers; ldq_i = lda_i
 *                          and ldr_i = n_i (Q_i may equal A_i)        (args 6-8)
 *   variant                as in cqr_factor                          (arg 9)
 *   status                 DEVICE int array of length batch: per-matrix
 *                          status codes as in cqr_factor              (arg 10)
 *   workspace, ws_bytes    >= cqr_batched_workspace_size(), or NULL
 *                          (registered allocator; synchronous)        (args 11, 12)
 *   stream                 CUDA stream                               (arg 13)
 * The host size arrays come first and the device-pointer arrays after
 * them; Q_i and R_i take the leading dimensions lda_i and n_i, so there are
 * no ldq / ldr arrays.
 * Either way the whole call is ordered on `stream`, reads no host memory
 * after it returns (the persistent path's descriptor table travels as
 * kernel parameters), and can be captured into a CUDA graph.  Calls that
 * share the workspace must not overlap on the GPU.
 */
int cqr_factor_batched(int batch, const int64_t* m, const int64_t* n, const int64_t* lda, const int* panel_b,
                       double* const* A, double* const* Q, double* const* R, int variant, int* status,
                       void* workspace, size_t ws_bytes, cqr_stream_t stream);

/*
 * cqr_test_arm_wait_expiry: test hook of the bounded waits (failure
 * detection; not in the paper).  Every mbarrier wait inside the tensor-core
 * kernels of CQR_EMULATED is bounded in time (2 s); on expiry the block
 * records CQR_STATUS_TIMEOUT in the status word, waits (bounded) for its
 * copies in flight, frees its tensor memory and returns, and every later
 * kernel of the call returns at once.  This hook makes that path run: the
 * NEXT launch of the chosen kernel withholds the copies of one stage, so
 * the waits for it expire after `wait_ns`, and the hook disarms itself.
 *   kernel   0 = the product kernel (Gram matrices, projections), 1 = the
 *            update kernel, -1 = disarm                              (arg 1)
 *   stage    first stage (per block) whose copies are withheld, >= 0  (arg 2)
 *   wait_ns  bound of every wait of that launch, 1 .. 2e9             (arg 3)
 * Host-side only (nothing is launched).  Returns 0, or -i for argument i.
 */
int cqr_test_arm_wait_expiry(int kernel, int stage, long long wait_ns);

/*
 * cqr_batched_panel_widths: after a persistent cqr_factor_batched call
 * (synchronises `stream`), copies each matrix's final panel width (its
 * last panel's, which CQR_HALVE may have narrowed) into the HOST array
 * panel_b[batch].  Returns 0, -1 (batch < 1), -2 (NULL workspace),
 * -4 (NULL panel_b) or CQR_ERR_CUDA.
 */
int cqr_batched_panel_widths(int batch, const void* workspace, cqr_stream_t stream, int* panel_b);

/*
 * cqr_test_arm_barrier_expiry: test hook of the persistent batched launch's
 * bounded group barriers (failure detection; not in the paper).  In the
 * NEXT persistent launch, CTA `rank` of group `group` skips its arrival at
 * its `barrier`-th group barrier (1-based) and every barrier wait of that
 * launch is bounded by `wait_ns`, so the other CTAs' waits expire; the
 * hook then disarms itself.  group = -1 disarms.  Host-side only.  Returns
 * 0, or -i for argument i.
 */
int cqr_test_arm_barrier_expiry(int group, int rank, int barrier, long long wait_ns);

/* cqr_status_string: static description of a status or return code. */
const char* cqr_status_string(int status);

/*
 * cqr_probe_fp64_peak: measures this GPU's FP64 FMA throughput (DFMA chains
 * on every SM, kind 0 of cqr_probe_fp64) for `iters` iterations and returns
 * GFLOP/s (<= 0 on error).  Synchronous.
 */
double cqr_probe_fp64_peak(int iters);

/*
 * cqr_probe_fp64: FP64 peak microbenchmarks, the denominators of the
 * roofline fractions (measurement support; not in the paper).
 *   kind   0 = DFMA on the CUDA cores (the pipe every native kernel here
 *          uses); 1 = FP64 tensor cores, mma.sync m8n8k4 .f64; 2 = FP64
 *          tensor cores, mma.sync m16n8k16 .f64                        (arg 1)
 *   iters  iterations of the timed loop (about 1e5 gives ~0.1 s)      (arg 2)
 *   gflops, flop_per_clk_sm, sm_mhz  HOST outputs (each may be NULL): the
 *          throughput of the fastest of three single-wave launches, its
 *          FLOPs per SM clock cycle (SM cycle counters, independent of the
 *          clock the GPU ran at) and the effective SM clock, cycles / time
 *                                                                  (args 3-5)
 * Synchronous, on the legacy default stream; allocates nothing.  Returns 0,
 * -1 for a bad kind, -2 for iters < 1, CQR_ERR_CUDA on a CUDA error.
 */
int cqr_probe_fp64(int kind, int iters, double* gflops, double* flop_per_clk_sm, double* sm_mhz);

/*
 * Launch accounting and kernel timing (measurement support; not in the
 * paper).  Kernel classes: 0 Gram (syrk partials), 1 projection (split-m
 * X^T Z partials), 2 split-m reduction, 3 Cholesky, 4 triangular solve,
 * 5 GEMM update (A -= Q Y, P -= Q Z, R products), 6 other kernels (adjoint
 * helpers, probes, the digit splitting of CQR_EMULATED), 7 batched
 * scheduler.
 *
 * cqr_launch_count: number of kernels this process has launched through the
 *   library so far (host counter; monotonic).
 * cqr_profile_enable: from now on, bracket every launch with a CUDA event
 *   pair on its stream (host-side event objects, created up front for
 *   `capacity` launches; later launches are not timed).  Clears earlier
 *   records.  Do not enable around a CUDA-graph capture.  Returns 0, -1 for
 *   capacity < 1, CQR_ERR_CUDA if events cannot be created.
 * cqr_profile_disable: stop recording (records are kept).
 * cqr_profile_read: synchronises on the recorded events and returns, for
 *   kernel class `cls`, the number of timed launches, their summed device
 *   time in ms, and their summed algorithmic FLOP counts (Gram m b (b+1),
 *   projection 2 m p q, Cholesky b^3/3, triangular solve m b^2, update
 *   2 M N K).  Returns 0, -1 for a bad argument, CQR_ERR_CUDA on error.
 * cqr_kernel_class_name: static name of a kernel class.
 */
/*
 * Tracing.  The enqueue of every call brackets its phases with NVTX ranges
 * (domain "cqr"; no cost unless a tool such as Nsight Systems is attached):
 *   mCQR2GS (Alg. 9), panel j = 0 .. k-1 (with CQR_HALVE: the panel's first
 *   column):  "cqr2_first_panel" 0 (step 1), then for j >= 1
 *   "project_update" (steps 3-5: Y = Q_{j-1}^T A_{j:k}, A_{j:k} -= Q_{j-1} Y),
 *   "cqr" (step 6), "reorthogonalise" (step 7), "cqr_final" (step 8),
 *   "r_update" (R_jj = S2 S1, R_{1:j-1,j} += Z S1); with CQR_HALVE each
 *   attempt of a panel's first CholeskyQR is "panel_test";
 *   CQR2GS (Alg. 7): "cqrgs_pass" 0 and 1 (Alg. 6 twice), each holding
 *   "cqr" j and "project_update" j per panel, then "r_update" -1;
 *   CholeskyQR2 / shifted CholeskyQR3: "cqr2" / "scqr3" with panel -1;
 *   cqr_factor_batched: "batched" with panel = batch size; cqr_backward:
 *   "backward" -1.
 * The ranges time the host-side enqueue (the kernels run asynchronously;
 * a tool correlates them with the launches inside each range).
 * cqr_set_trace(fn, ctx): also call fn(phase, panel, begin, ctx) on the
 *   enqueueing thread at the start (begin = 1) and end (begin = 0) of every
 *   phase; fn = NULL unregisters.  fn runs while the call may hold the
 *   library's per-device stream locks, so it must not call the library (it
 *   may record CUDA events, as a timeline tool does).  Returns 0.
 */
typedef void (*cqr_trace_fn)(const char* phase, int panel, int begin, void* ctx);
int cqr_set_trace(cqr_trace_fn fn, void* ctx);

unsigned long long cqr_launch_count(void);
int cqr_profile_enable(int capacity);
int cqr_profile_disable(void);
int cqr_profile_read(int cls, long long* launches, double* total_ms, double* flops);
const char* cqr_kernel_class_name(int cls);

#ifdef __cplusplus
}
#endif

#endif /* CQR_GB300_H */
