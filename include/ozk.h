/*
 * ozk.h -- C ABI of the GB300 (sm_103a) emulated-ZGEMM / KKR tau_00 library (libozk.so).
 *
 * Method: the Ozaki-I scheme the paper uses to run FP64 GEMMs on low-precision tensor
 * cores (Sec. 2.2: split high-precision matrices into low-precision slices by significant
 * bits with exponent alignment, multiply slice pairs, accumulate in higher precision;
 * Sec. 3.2 and Sec. 4: the precision knob is a mantissa-bit count, 31..63 bits), applied
 * to ZGEMM and to the LU-based inversion of the KKR multiple scattering matrix that
 * dominates the LSMS method (Sec. 3.2).
 *
 * Reading used throughout (identical in the CPU oracle):
 *   - S slices of 8 bits each carry B = 8S - 1 fixed-point bits per row (columns for the
 *     right operand): e_i = frexp exponent of max_l max(|Re a_il|, |Im a_il|),
 *     X = trunc(x 2^(B - e_i)), X = sum_t d_t 256^(S-t) with balanced digits
 *     (d_t in [-128, 127] for t >= 2, d_1 in [-128, 128]).
 *   - Complex operands use the 4M stacked form: [Re A | Im A] times, per output column j,
 *     the rows [Re B_j ; -Im B_j] and [Im B_j ; Re B_j].
 *   - Slice pairs (s, t) with s + t <= S + 1 ("triangular", default) or all S x S ("full").
 *     Their products are exact integers (held as fp16 values on the sm_103a tensor cores,
 *     accumulated exactly in FP32, combined exactly in 128-bit integers).
 *   - The result 2^(e_i + f_j - 2B) sum_g G_g 256^(2S - g) is rounded once to binary64.
 *
 * Conventions
 *   - Matrices are complex binary64 ("double complex", interleaved re, im) in COLUMN-MAJOR
 *     order with a leading dimension, as in BLAS ZGEMM.  Pointers to matrices are DEVICE
 *     pointers owned by the caller; pointer arrays of batched calls are DEVICE arrays;
 *     per-problem size arrays of batched calls are HOST arrays.
 *   - Every call is asynchronous on the handle's stream (ozk_set_stream) and returns as
 *     soon as the work is enqueued.  Argument errors are reported synchronously by the
 *     return value and nothing is enqueued.  Errors detected on the device (non-finite
 *     input, singular pivot block, timed-out wait) set bits in a device status word that
 *     ozk_get_status() reads (after synchronising the stream) and clears.
 *   - Workspace (slice buffers, exponents, pivot inverses) is owned by the handle and
 *     grown on demand with cudaMalloc; ozk_reserve() sizes it up front so that later calls
 *     (for example inside a CUDA graph capture) never allocate.  A call that would need to
 *     grow the workspace while its stream is being captured returns OZK_ERR_CAPTURE.
 *   - Stream capture: a call may be captured into a CUDA graph once a call with the same
 *     sizes has run on the handle outside capture.  That call sizes the workspace and copies
 *     the host size arrays of batched calls to device memory, where the handle keeps each
 *     distinct array until it is destroyed (up to 4096 of them; the 4097th empties the
 *     cache).  Sizes first seen during capture return OZK_ERR_CAPTURE.  A captured graph
 *     holds the workspace and size-table addresses: it stays valid while the handle lives,
 *     its workspace does not grow and its size cache is not emptied, and its replays must
 *     not overlap other work that uses the same handle.  The launch profiler does not time
 *     captured launches.
 *   - Nothing aborts the process.
 */
#ifndef OZK_H
#define OZK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OZK_OK = 0,
    OZK_ERR_ARG = 1,        /* invalid argument (sizes, leading dimensions, S, mode) */
    OZK_ERR_NONFINITE = 2,  /* device flag: a NaN or Inf operand was met */
    OZK_ERR_SINGULAR = 3,   /* device flag: an exactly singular pivot block */
    OZK_ERR_TIMEOUT = 4,    /* device flag: a bounded device-side wait gave up */
    OZK_ERR_CUDA = 5,       /* a CUDA runtime call failed (message: ozk_last_error) */
    OZK_ERR_RANGE = 6,      /* the exact integer sum could exceed 128 bits for this S, k */
    OZK_ERR_CAPTURE = 7,    /* workspace growth needed during stream capture */
    OZK_ERR_RESIDUAL = 8,   /* a-posteriori residual check failed and fallback disabled */
    OZK_ERR_NOFILE = 9      /* file could not be read or written */
} ozk_status_t;

/* pair-set modes */
#define OZK_PAIRS_TRI 0
#define OZK_PAIRS_FULL 1

typedef struct ozk_context* ozk_handle_t;

/* ---- handle ------------------------------------------------------------------------ */

/* Create a handle on the current CUDA device.  Allocates the device status word. */
ozk_status_t ozk_create(ozk_handle_t* handle);
/* Destroy a handle and free its workspace (synchronises its stream first). */
ozk_status_t ozk_destroy(ozk_handle_t handle);
/* Stream (a cudaStream_t passed as void*; NULL = legacy default stream) for later calls. */
ozk_status_t ozk_set_stream(ozk_handle_t handle, void* stream);
/* Synchronise the stream, return the accumulated device status (0 or a bitwise OR of
 * 1 << OZK_ERR_* codes) in *device_flags and clear it.  Returns OZK_ERR_CUDA on a CUDA
 * error, else OZK_OK. */
ozk_status_t ozk_get_status(ozk_handle_t handle, int* device_flags);
/* Grow the handle's workspace to at least `bytes` now (never shrinks). */
ozk_status_t ozk_reserve(ozk_handle_t handle, size_t bytes);
/* Workspace bytes that ozaki_zgemm needs for (m, n, k, S, batch). */
size_t ozk_zgemm_workspace_size(int m, int n, int k, int S, int batch);
/* Message of the last OZK_ERR_CUDA / OZK_ERR_ARG on this thread (static storage). */
const char* ozk_last_error(void);
/* Number of kernel launches this library has enqueued on this thread so far. */
uint64_t ozk_launch_count(void);

/* ---- launch profiler ---------------------------------------------------------------- */

/* Kernel kinds reported by ozk_profile_end (array index). */
#define OZK_KIND_SPLIT 0       /* exponent scan + slice split */
#define OZK_KIND_SLICE_GEMM 1  /* tcgen05 slice-pair GEMM + reconstruction */
#define OZK_KIND_GJ 2          /* pivot-block Gauss-Jordan inverse / solve */
#define OZK_KIND_BUILD_M 3     /* M = I - t G */
#define OZK_KIND_DMMA 4        /* binary64 DMMA ZGEMM */
#define OZK_KIND_OTHER 5
#define OZK_KERNEL_KINDS 6

/* Start recording a CUDA event pair on the handle's stream around every launch (no
 * synchronisation; negligible overhead), clearing earlier records. */
ozk_status_t ozk_profile_begin(ozk_handle_t handle);
/* Stop recording, synchronise, and return per kind (arrays of OZK_KERNEL_KINDS entries):
 * launches, summed device milliseconds, summed algorithmic flops (slice GEMM: integer
 * multiply-adds x 2 of all slice pairs, P_S 8 m n k; DMMA: 8 m n k) and algorithmic bytes. */
ozk_status_t ozk_profile_end(ozk_handle_t handle, uint64_t* launches, double* ms, double* flops,
                             double* bytes);
/* Per kind (OZK_KERNEL_KINDS entries), the bytes the kernels of the last ozk_profile_end window
 * read and wrote in this library's storage layout, beside the algorithmic `bytes` of that call:
 * the split's algorithmic figure counts int8 digits (2S bytes per left-operand element, 3S per
 * right-operand element: Re, Im, -Im), while the fp16-held planes move 4S and 8S. */
ozk_status_t ozk_profile_moved(ozk_handle_t handle, double* moved);

/* ---- emulated ZGEMM (paper Sec. 2.2, Sec. 3.2) ------------------------------------ */

/* C = alpha op(A) op(B) + beta C with op(X) in {'N', 'T', 'C'} (none, transpose,
 * conjugate transpose), exactly the BLAS ZGEMM argument list plus the slice count S.
 *   alpha, beta : HOST pointers to two doubles (re, im).
 *   A, B, C     : DEVICE pointers, column major, lda/ldb/ldc >= rows of the stored matrix.
 *   S           : 1..16 slices (B = 8S - 1 bits); 0: the slice-count selector chooses S
 *                 in 3..10 and checks the result (see the selector section; triangular pairs);
 *                 < 0: the binary64 DMMA GEMM (ozk_zgemm_dmma, pair_mode ignored).  The same
 *                 rule holds for every S argument of this library.
 *                 pair_mode: OZK_PAIRS_TRI / _FULL.
 * Epilogues: beta == 0 stores RN(alpha Z) (alpha == 1: bitwise equal to the oracle);
 * alpha == -1, beta == 1 computes C - RN(Z) with one binary64 subtraction (bitwise equal
 * to the oracle's LU update); other alpha, beta use binary64 complex arithmetic.
 * k == 0 or alpha == 0 scales C by beta.  Returns OZK_ERR_RANGE if 8(g_max - 2) + 14 +
 * log2(2k * S) + 2 > 127 (the exact 128-bit sum could overflow). */
ozk_status_t ozaki_zgemm(ozk_handle_t handle, char transa, char transb, int m, int n, int k,
                         const double* alpha, const void* A, int lda, const void* B, int ldb,
                         const double* beta, void* C, int ldc, int S, int pair_mode);

/* Batched form: `batch` independent problems; A, B, C are DEVICE arrays of `batch` DEVICE
 * pointers; m, n, k, lda, ldb, ldc are HOST arrays of `batch` entries (variable sizes).
 * Problems with m, n == 0 are skipped.  S >= 1 emulated, S < 0 binary64 DMMA over the same
 * tables; S = 0 (the selector, a single-GEMM mode) returns OZK_ERR_ARG. */
ozk_status_t ozaki_zgemm_vbatched(ozk_handle_t handle, char transa, char transb,
                                  const int* m, const int* n, const int* k,
                                  const double* alpha, const void* const* A, const int* lda,
                                  const void* const* B, const int* ldb, const double* beta,
                                  void* const* C, const int* ldc, int batch, int S, int pair_mode);

/* Allocation-free emulated ZGEMM (no counterpart in the paper: an interface for callers that
 * cannot allocate device memory when they call -- for example code running inside a CUDA
 * graph capture, where cudaMalloc is not allowed, or inside a framework whose memory pool
 * forbids allocations it does not own).  Same arguments and results as ozaki_zgemm, but with
 * no handle: `stream` is a cudaStream_t (NULL = legacy default stream) and the scratch is a
 * static device array of OZK_NOALLOC_SCRATCH_BYTES compiled into the library, so nothing is
 * allocated.  Every GPU that loads the library holds that array until the process exits.
 *   - The first call on each device looks up the array's device address with
 *     cudaGetSymbolAddress (once per device, with that device current); make that first call
 *     before any stream capture.
 *   - Problems whose scratch (ozk_zgemm_workspace_size) exceeds OZK_NOALLOC_SCRATCH_BYTES are
 *     rejected with OZK_ERR_ARG before anything is enqueued.
 *   - All calls share the array and it keeps the last call's contents (each call rewrites
 *     what it reads); calls that may overlap on the GPU race and must be serialised.
 *   - device_status: DEVICE int that collects OZK_ERR_* bits as in ozk_get_status (the caller
 *     clears and reads it); NULL uses a flag inside the library that nobody reads. */
#define OZK_NOALLOC_SCRATCH_BYTES (32u << 20)
ozk_status_t ozaki_zgemm_noalloc(void* stream, char transa, char transb, int m, int n, int k,
                                 const double* alpha, const void* A, int lda, const void* B, int ldb,
                                 const double* beta, void* C, int ldc, int S, int pair_mode,
                                 int* device_status);

/* ---- slice-count selector -------------------------------------------------------------
 *
 * The paper finds that accuracy depends on the precision and on the operator and handles it
 * by tuning the precision (Abstract; Sec. 4 shows the error falling mode by mode; Sec. 5
 * argues for adaptive precision); it gives no rule for choosing S.  This library's selector:
 *   1. computes 16 features of op(A) op(B) (ozk_selector_features; definitions in
 *      csrc/selector.cu) from per-row / per-column statistics and a probe product
 *      z = op(A) (op(B) X), X = 2 counter-based random probe vectors;
 *   2. predicts log10 of the relative Frobenius error for S = 3..10 with a float32
 *      perceptron 16 -> 64 -> 64 -> 8 (ReLU), whose parameters are trained on the GPU by
 *      ozk_selector_train_step (mean squared error, Adam);
 *   3. picks the smallest S whose prediction is <= log10(tol) - margin (else 10);
 *   4. checks the computed product D a posteriori: r = ||D X - z|| / ||z|| (4 probe vectors,
 *      compensated double-double products) estimates ||D - AB||_F / ||AB||_F; if r > tol / 2
 *      (room for the estimate's scatter) the product is recomputed with S = 10 (fallback),
 *      unless OZK_SEL_NO_FALLBACK is set, in which case OZK_ERR_RESIDUAL is returned.
 * ozaki_zgemm with S = 0 runs these steps.  It synchronises the stream twice (to read the
 * chosen S and the residual) and cannot be captured (OZK_ERR_CAPTURE).  Parameter layout,
 * OZK_SEL_NPARAMS floats: W1[64][16], b1[64], W2[64][64], b2[64], W3[8][64], b3[8]. */
#define OZK_SEL_FEATURES 16
#define OZK_SEL_OUTPUTS 8
#define OZK_SEL_NPARAMS 5768
#define OZK_SEL_SMIN 3
#define OZK_SEL_SMAX 10
#define OZK_SEL_NO_FALLBACK 1

typedef struct {
    int S_selected;            /* S chosen from the prediction */
    int S_used;                /* S of the returned product (S_selected or OZK_SEL_SMAX) */
    int fallback;              /* 1 if the product was recomputed with OZK_SEL_SMAX */
    int residual_ok;           /* 1 if the returned product passed the residual check */
    double residual;           /* residual estimate of the returned product */
    double residual_selected;  /* residual estimate of the product at S_selected */
    float predicted_log10_err[OZK_SEL_OUTPUTS];   /* for S = 3..10 */
    uint64_t probe_seed;       /* seed of the probe vectors of this call */
    int gemms;                 /* kkr_tau00 (S = 0): GEMMs of the solve; ozaki_zgemm: 0 */
    int S_count[OZK_SEL_OUTPUTS];                 /* kkr_tau00 (S = 0): GEMMs chosen at S = 3..10 */
} ozk_selector_info;

/* Random initial parameters (He-scaled normals from a counter-based generator seeded by
 * `seed`, zero biases); resets the Adam state. */
ozk_status_t ozk_selector_init(ozk_handle_t handle, uint64_t seed);
/* Copy parameters from / to a HOST array of OZK_SEL_NPARAMS floats (set resets Adam). */
ozk_status_t ozk_selector_set_params(ozk_handle_t handle, const float* params);
ozk_status_t ozk_selector_get_params(ozk_handle_t handle, float* params);
/* Parameter file: 8 bytes "OZKSEL1\0", int32 OZK_SEL_NPARAMS, then the floats (little
 * endian).  OZK_ERR_NOFILE if it cannot be read or written, OZK_ERR_ARG if malformed. */
ozk_status_t ozk_selector_load(ozk_handle_t handle, const char* path);
ozk_status_t ozk_selector_save(ozk_handle_t handle, const char* path);
/* Tolerance on the relative Frobenius error (default 1e-10), safety margin in decades
 * subtracted from log10(tol) when choosing (default 0.6: the check passes a product whose
 * estimate is at most tol / 2, and the 4-probe estimate scatters around the true error, so
 * the choice aims at tol / 4 for a product whose error is as predicted to pass), flags
 * (OZK_SEL_NO_FALLBACK). */
ozk_status_t ozk_selector_configure(ozk_handle_t handle, double tol, double margin, int flags);
/* The 16 features of op(A) op(B) into a DEVICE array of 16 floats, with the probe vectors
 * of `probe_seed`.  k >= 1. */
ozk_status_t ozk_selector_features(ozk_handle_t handle, char transa, char transb, int m, int n, int k,
                                   const void* A, int lda, const void* B, int ldb, uint64_t probe_seed,
                                   float* features);
/* Y (N x 8) = perceptron(X (N x 16)); DEVICE row-major float arrays. */
ozk_status_t ozk_selector_predict(ozk_handle_t handle, int N, const float* X, float* Y);
/* One Adam step (lr; beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error of the
 * predictions of X (N x 16) against targets T (N x 8), DEVICE row-major float arrays.
 * *loss (HOST, may be NULL) receives the loss before the step (synchronises the stream). */
ozk_status_t ozk_selector_train_step(ozk_handle_t handle, int N, const float* X, const float* T, float lr,
                                     double* loss);
/* Gradient of that loss with respect to the parameters, into a DEVICE array of
 * OZK_SEL_NPARAMS floats, without updating them. */
ozk_status_t ozk_selector_gradient(ozk_handle_t handle, int N, const float* X, const float* T, float* grad);
/* Training-data log of the selector: while active, every S = 0 GEMM on this handle (ozaki_zgemm
 * and the GEMMs of kkr_tau00 with S = 0) also writes one row of its 16 features (DEVICE array
 * `features`, 16 floats per row) and of the log10 relative Frobenius errors of its products at
 * S = 3..10 against the S = 12 product, floored at -17 (DEVICE array `targets`, 8 floats per
 * row), up to `capacity` rows; later GEMMs are not recorded.  Each logged GEMM runs nine extra
 * emulated products.  ozk_selector_log_end stops logging, synchronises and returns the number
 * of rows written. */
ozk_status_t ozk_selector_log_begin(ozk_handle_t handle, float* features, float* targets, int capacity);
ozk_status_t ozk_selector_log_end(ozk_handle_t handle, int* count);
/* What the last S = 0 call on this handle (ozaki_zgemm, kkr_tau00 or a batched solve) chose
 * and measured. */
ozk_status_t ozk_selector_last(ozk_handle_t handle, ozk_selector_info* info);
/* ||X - Y||_F / ||Y||_F of two m x n DEVICE matrices (column major) into *rel (HOST);
 * synchronises the stream. */
ozk_status_t ozk_rel_diff(ozk_handle_t handle, int m, int n, const void* X, int ldx, const void* Y, int ldy,
                          double* rel);

/* Ozaki-II (CRT) emulated ZGEMM (paper Sec. 2.2: integers, products modulo small pairwise-
 * coprime moduli, Chinese-Remainder reconstruction; precision knob: the number of moduli,
 * Sec. 3.2).  Same arguments as ozaki_zgemm with nmod (2..16) in place of S.  Moduli: the nmod
 * largest pairwise-coprime integers <= 256; integer images trunc(x 2^(beta - e)) with per-row
 * (per-column) frexp exponents e and beta the largest bit count with 2k 4^beta < P/2 (P the
 * product of the moduli), so the exact product is recovered; one rounding to binary64.  The
 * residue products run on the tcgen05 tensor cores (one product per modulus, exact integers
 * added to an int32 buffer of nmod x m x 2n in the workspace), the reconstruction in a separate
 * kernel.  k <= 65536. */
ozk_status_t ozaki2_zgemm(ozk_handle_t handle, char transa, char transb, int m, int n, int k,
                          const double* alpha, const void* A, int lda, const void* B, int ldb,
                          const double* beta, void* C, int ldc, int nmod);

/* Plain binary64 ZGEMM on the FP64 tensor path (DMMA, mma.sync m8n8k4.f64), same argument
 * meaning as ozaki_zgemm without S: the comparison baseline on the same GPU. */
ozk_status_t ozk_zgemm_dmma(ozk_handle_t handle, char transa, char transb, int m, int n, int k,
                            const double* alpha, const void* A, int lda, const void* B, int ldb,
                            const double* beta, void* C, int ldc);

/* ---- test hooks for the individual steps ---------------------------------------- */

/* Exponent scan + split of op(X) as the LEFT operand (side 0: rows of op(A)) or as the
 * RIGHT operand (side 1: columns of op(B)).  op(X) has `rows` rows of length k (side 0) or
 * is k x rows (side 1).  Outputs (DEVICE): exps[rows] (int32) and digits as int16
 * [S][rows'][2k] with rows' = rows (side 0) or 2 rows (side 1, stacked layout). */
ozk_status_t ozk_split_debug(ozk_handle_t handle, int side, char trans, int rows, int k,
                             const void* X, int ldx, int S, int32_t* exps, int16_t* digits);
/* Exact group sums G_g (int64 [G][m][2n], g = 2 .. g_max) of the slice-pair products
 * for C = op(A) op(B), computed by the tensor-core kernel (the emulated GEMM with its
 * reconstruction replaced by an integer dump).  DEVICE output. */
ozk_status_t ozk_group_sums_debug(ozk_handle_t handle, char transa, char transb, int m, int n,
                                  int k, const void* A, int lda, const void* B, int ldb, int S,
                                  int pair_mode, int64_t* groups);

/* Failure-path hook of the bounded device waits (the paper has no counterpart; every wait of
 * the tensor-core kernel is bounded so that a lost arrival cannot hang the GPU).  The next
 * slice-GEMM launch enqueued on this handle first makes one thread of every CTA wait on a
 * barrier that no thread ever arrives at, with a budget of `cycles` SM clock cycles, before the
 * CTA has issued any TMA copy or MMA.  The wait gives up, sets OZK_ERR_TIMEOUT in the device
 * status word, and the CTA skips its tiles, releases its tensor memory and exits: that GEMM
 * leaves its output unwritten.  The launch after it runs normally.  cycles <= 0 clears a pending
 * request. */
ozk_status_t ozk_debug_stall_next_gemm(ozk_handle_t handle, long long cycles);

/* ---- KKR tau_00 (paper Sec. 3.2) ----------------------------------------------------- */

/* M = I - t G for a LIZ of L sites with b x b blocks (n = L b).
 *   t : DEVICE, L blocks of b x b, block l at t + l*b*b, each column major (ld b).
 *   G : DEVICE, n x n column major (ld n).  M: DEVICE, n x n column major (ld n). */
ozk_status_t kkr_build_m(ozk_handle_t handle, int L, int b, const void* t, const void* G, void* M);

/* Batched M_z = I - t_z G_z for `batch` LIZs of L[z] sites (HOST array) with b x b blocks;
 * t, G, M are DEVICE arrays of DEVICE pointers with the layouts of kkr_build_m.  Several
 * entries may share one G (atoms of one lattice at one energy). */
ozk_status_t kkr_build_m_batched(ozk_handle_t handle, int batch, const int* L, int b,
                                 const void* const* t, const void* const* G, void* const* M);

/* M_a = I - blockdiag(t_a) G for natoms atoms that share one G (atoms of one lattice at one
 * energy), every product an emulated GEMM with S slices (paper Sec. 3.2: the KKR matrix is
 * built by the ZGEMMs the emulation intercepts).  For each site block row i the atoms' blocks
 * t_{a,i} are stacked into one (natoms b) x b left operand and multiplied by the block row
 * G[ib:(i+1)b, :] in one GEMM (L GEMMs in one launch); the epilogue writes I - RN(Z) straight
 * into the atoms' M (row a b + r of GEMM i is row i b + r of M_a), reading no C.
 *   t: DEVICE array of natoms DEVICE pointers, each to L column-major b x b blocks (block l
 *      at offset l b b).  G: DEVICE n x n column major (n = L b).  M: DEVICE array of natoms
 *      DEVICE pointers to n x n column-major outputs (ld n). */
ozk_status_t kkr_build_m_shared(ozk_handle_t handle, int natoms, int L, int b, const void* const* t,
                                const void* G, void* const* M, int S);
/* The same for atoms whose LIZs are the first L[a] sites (HOST array) of one site list on one
 * lattice at one energy: atom a's G is the leading L[a] b block of G (the structure constants
 * of the largest LIZ, leading dimension ldg >= max L[a] b), its M has order and leading
 * dimension L[a] b, and t[a] holds L[a] blocks.  One stacked GEMM per block row i < max L[a];
 * the rows of atoms with L[a] <= i, and columns past an atom's order, are not written. */
ozk_status_t kkr_build_m_shared_sizes(ozk_handle_t handle, int natoms, const int* L, int b,
                                      const void* const* t, const void* G, int ldg, void* const* M, int S);

/* tau_00 = [M^-1]_00 t_0 = S_00^-1 t_0 by block LU (paper Sec. 3.2: LU-based inversion of the
 * multiple scattering matrix).  Panels J = [p, q) of width nb are eliminated from the trailing
 * end of M, so the centre block (site 0, rows/cols 0..b-1) is eliminated last and S_00 is the
 * Schur complement left there.
 * Each panel: D^-1 of its pivot block D = M[p:q, p:q] (in-place Gauss-Jordan with partial
 * pivoting in binary64), L = M[0:p, p:q] D^-1 written in place, M[0:p, 0:p] -= L M[p:q, 0:p].
 * The operation on (t, G, LIZ) is kkr_build_m (or kkr_build_m_shared for atoms sharing G)
 * followed by this call on the M it built.  The slice count follows the ozaki_zgemm rule:
 *   S >= 1: both GEMMs are the emulated ZGEMM with S slices.
 *   S = 0:  every GEMM is the emulated ZGEMM at the slice count the selector picks for its
 *           operands (one stream synchronisation per GEMM to read the choice), followed by
 *           the probe residual check of ozaki_zgemm (S = 0), recorded on the device.  The
 *           record is read once when the solve ends; if any check failed, M is restored from
 *           a copy taken at the start (n x n in the workspace) and the solve is redone with
 *           every GEMM at S = 10, again checked (OZK_SEL_NO_FALLBACK: no copy, and a failed
 *           check returns OZK_ERR_RESIDUAL).  Needs selector parameters; cannot be captured.
 *           ozk_selector_last reports the solve: the largest S chosen (S_selected), the GEMMs
 *           per S (S_count), the largest residual estimate, and whether it was redone.
 *   S < 0:  both GEMMs are binary64 DMMA GEMMs (the native-precision baseline).
 *   nb <= OZK_NB_MAX (the pivot block is held in shared memory).  nb = 0: for S >= 1 the
 *   (W, w) pair kkr_tau00_autotune_panels picks for one matrix of order n (tuned on the first
 *   such call, which must not be captured, and cached in the handle); with leaves (w < W) the
 *   solve is the one-matrix case of kkr_tau00_batched_panels (leaves narrower than the panels
 *   cut the binary64 pivot-inverse work, which runs on one SM per inverse for a single
 *   matrix), with whole panels (w = W) this path with nb = W.  S = 0 takes the whole-panel width kkr_tau00_autotune picks at S = 7; S < 0, 32.
 *   M   : DEVICE n x n column major (ld n), DESTROYED (overwritten by the factorisation).
 *   t0  : DEVICE b x b column major.  tau00: DEVICE b x b column major output.
 *   b <= 64 (16 for lmax = 3; 50 for lmax = 4 with spin), nb a multiple of b.  Site 0 occupies
 *   rows/cols 0..b-1; the final S_00^-1 t_0 is a Gauss-Jordan solve (a 4-warp kernel up to
 *   16 x 16, a 256-thread one above). */
#define OZK_NB_MAX 112            /* largest pivot-block (leaf) width of the tau_00 solves */
#define OZK_PANEL_MAX 448         /* largest panel width of kkr_tau00_batched_panels */
ozk_status_t kkr_tau00(ozk_handle_t handle, int n, int b, void* M, const void* t0, void* tau00,
                       int S, int nb);

/* Right-side triangular solve with emulated GEMMs (paper Sec. 3.2: the ZGEMM and ZTRSM mix of
 * the LU-based inversion): solves X T = B for X and overwrites B with it.  T: DEVICE n x n
 * column major (ld ldt >= n), upper (uplo 'U') or lower ('L') triangular, its stored diagonal
 * used (diag 'N') or taken as ones ('U'); the other triangle is not read.  B: DEVICE m x n
 * column major (ld ldb >= m).  Block columns of 16: each block column of X is B's block column
 * minus the already solved columns times T's block column (an emulated GEMM with S slices),
 * times the binary64 inverse of T's 16 x 16 diagonal block (an emulated GEMM).  A zero
 * diagonal element of a non-unit T sets OZK_ERR_SINGULAR.  S in 1..16. */
ozk_status_t ozaki_ztrsm(ozk_handle_t handle, char uplo, char diag, int m, int n, const void* T, int ldt,
                         void* B, int ldb, int S);

/* tau_00 as kkr_tau00, with every pivot block factored instead of inverted: P D = L U (binary64,
 * partial pivoting; the row interchanges are applied to the panel's row strip too), then
 * M_RJ := M_RJ U^-1 L^-1 by two emulated ZTRSMs (ozaki_ztrsm) and M_RR -= M_RJ (P M_JR) by an
 * emulated GEMM.  Arguments as kkr_tau00 (nb >= b explicit, S >= 1). */
ozk_status_t kkr_tau00_lu(ozk_handle_t handle, int n, int b, void* M, const void* t0, void* tau00,
                          int S, int nb);

/* Batched tau_00 over `nsolves` independent (atom, energy) matrices of sizes n[i] (HOST
 * array, multiples of b): M, t0, tau00 are DEVICE arrays of DEVICE pointers.  All solves
 * advance panel by panel in lockstep; each step is one batched launch per kernel.
 * nb = 0: the panel and leaf widths an autotuner chose for these sizes, b and S (a cached
 * kkr_tau00_autotune or kkr_tau00_autotune_panels result; without one, the latter runs on the
 * first such call, which must not be captured); see kkr_tau00_batched_panels.
 * S = 0: one slice count serves every launch of the call (a launch covers all solves), so the
 * selector picks S for the leading block (at most 512 x 512 outputs) of the first trailing
 * update (the L and U panels of the unfactored M) of up to 8 sampled solves (the largest, the
 * smallest and solves spread over the call) and the call takes the largest pick; each sampled product is then computed at that S and checked
 * with the probes, and a failed check sends the whole call to S = 10 (OZK_SEL_NO_FALLBACK:
 * OZK_ERR_RESIDUAL).  ozk_selector_last reports the choice, the sample size (gemms) and the
 * largest residual estimate.  Synchronises once per sampled solve.  S < 0: every GEMM in binary64 on the DMMA kernel (the native-precision baseline of
 * the same batched algorithm; L = M_RJ D^-1 goes to per-solve scratch in the handle's
 * workspace; nb = 0 means 32, as in kkr_tau00). */
ozk_status_t kkr_tau00_batched(ozk_handle_t handle, int nsolves, const int* n, int b,
                               void* const* M, const void* const* t0, void* const* tau00,
                               int S, int nb);

/* The same batched tau_00 with panels of width W (a multiple of b, <= OZK_PANEL_MAX) factored
 * leaf by leaf (paper Sec. 3.2's LU-based inversion with each panel's trailing update
 * deferred): the leaves [a, hi) of width w (a multiple of b, <= OZK_NB_MAX; the front leaf of a
 * panel narrower when w does not divide its width) are taken from the panel's end; per leaf
 * the binary64 inverse of its pivot block, L = M[0:a, a:hi] D^-1 in place and the update of
 * the frame of [0, a) x [0, a) outside [0, p) x [0, p) (emulated GEMMs with k = w); per panel
 * [p, q) one deferred update M[0:p, 0:p] -= M[0:p, p:q] M[p:q, 0:p], an emulated GEMM with
 * k = q - p.  In exact arithmetic this is the block LU of kkr_tau00_batched; the pivot blocks
 * stay w wide (the binary64 work of whole panels of width w) while the dominant updates get
 * W-deep products.  w = 0 or w = W: one leaf per panel (kkr_tau00_batched with nb = W).
 * W = 0: the (W, w) pair kkr_tau00_autotune_panels picks for these sizes, b and S (tuned on
 * the first such call, which must not be captured, and cached).  S as kkr_tau00_batched; the
 * binary64 DMMA form (S < 0) needs w = W. */
ozk_status_t kkr_tau00_batched_panels(ozk_handle_t handle, int nsolves, const int* n, int b,
                                      void* const* M, const void* const* t0, void* const* tau00,
                                      int S, int W, int w);

/* Contour-integrated observable of the tau_00 blocks of the energy points z_i of a contour:
 * traces[i] = Tr tau_00(z_i) and *integral = sum_i w_i Tr tau_00(z_i) (the quadrature of the
 * site-diagonal Green's-function trace whose error per precision mode the paper reports,
 * Sec. 4).  tau: DEVICE array of nsolves DEVICE pointers to b x b column-major blocks;
 * w: HOST 2 nsolves doubles (re, im of the weights); traces (HOST, 2 nsolves doubles, may
 * be NULL) and integral (HOST, 2 doubles).  Synchronises the stream. */
ozk_status_t kkr_contour_trace(ozk_handle_t handle, int nsolves, int b, const void* const* tau, const double* w,
                               double* traces, double* integral);

/* Autotuner of the batched solve: times kkr_tau00_batched on scratch matrices of the sizes
 * n[0..nsolves-1] (diagonally dominant test matrices, allocated and freed here) for every
 * panel width nb = b, 2b, ... <= OZK_NB_MAX, returns in *nb_best (HOST) the smallest nb among
 * those within 1 % of the fastest, and the times in
 * ms in times[] (HOST, one per candidate in that order; may be NULL), and caches the choice in
 * the handle for nb = 0.  Synchronises; cannot be captured. */
ozk_status_t kkr_tau00_autotune(ozk_handle_t handle, int nsolves, const int* n, int b, int S, int* nb_best,
                                float* times);

/* Autotuner over (W, w) pairs of kkr_tau00_batched_panels: whole-panel pivot blocks W = w = b,
 * 2b, ... <= OZK_NB_MAX, then panels of g leaves (W = g w <= OZK_PANEL_MAX, g = 2..4; g = 2..8
 * for nsolves = 1) for every leaf width w (a multiple of b) from 32 to 96.  Times each on
 * scratch test matrices of the sizes n[] as kkr_tau00_autotune does, returns in *W_best,
 * *w_best the smallest pair (by W, then w) among those within 1 % of the fastest and caches it
 * for W = 0 (and nb = 0 of kkr_tau00_batched).  Optional HOST outputs: times[] (ms) and cand[]
 * (W, w per candidate), each with room for `cap` candidates (OZK_ERR_ARG if too short; the
 * count is written to *ncand when ncand is not NULL). */
ozk_status_t kkr_tau00_autotune_panels(ozk_handle_t handle, int nsolves, const int* n, int b, int S,
                                       int* W_best, int* w_best, float* times, int* cand, int cap,
                                       int* ncand);

#ifdef __cplusplus
}
#endif
#endif /* OZK_H */
