// Kernel parameter blocks and launchers shared by the translation units of libozk.
#pragma once

#include "ozk_internal.cuh"

namespace ozk {

// ---- split.cu: exponent scan + balanced-digit slices
struct SplitParams {
  const double2* const* X;  // per problem: base pointer of the stored matrix (device)
  const int* ld;            // per problem: leading dimension (complex elements)
  const int* rows;          // per problem: logical rows (rows of op(A) / columns of op(B))
  const int* kdim;          // per problem: K
  int trans;                // logical X[r][l] = trans ? P[l + r ld] : P[r + l ld]
  int conj;                 // negate the imaginary part (op = 'C')
  int side;                 // 0 left operand, 1 right operand
  int S;
  int nbits;                // B = 8S - 1
  long long out_rows;       // row count of one slice plane
  long long kpad;           // row pitch (fp16 elements)
  __half* out;              // [batch][S][out_rows][kpad]
  int* exps;                // [batch][exp_stride]
  long long exp_stride;
  int16_t* dbg_digits;      // optional int16 copy [S][out_rows][2k] for problem 0 (test hook)
  int* status;
  // single-problem values, used when X == nullptr (no device tables needed); problem z of a
  // uniform batch starts at X1 + z * zstride1
  const double2* X1; int ld1, rows1, k1;
  long long zstride1;
  // K-parallel split (operands with few row blocks and long rows): gmax[z exp_stride + r] holds
  // the bit pattern of row r's largest |Re|, |Im| (taken by split_rowmax_kernel over K
  // segments), and kgroups CTAs share each row block's K tiles; kgroups <= 1: one CTA per row
  // block scans and splits the whole row
  unsigned long long* gmax;
  int kgroups;
};
struct SplitPair { SplitParams s[2]; int nsides; };

// ---- ozaki2.cu: Ozaki-II (CRT) residues, products and reconstruction
constexpr int OZ2_MAXMOD = 16;
struct Oz2Tables {
  int N;                         // number of moduli
  int mod[OZ2_MAXMOD];           // m_t
  int pow256[OZ2_MAXMOD][8];     // 256^s mod m_t
  int pm[OZ2_MAXMOD][OZ2_MAXMOD];   // (m_0 ... m_{j-1}) mod m_t, j < t (Garner)
  int inv[OZ2_MAXMOD];           // (m_0 ... m_{t-1})^-1 mod m_t
  unsigned long long P_lo, P_hi; // P = prod m_t (< 2^128)
};
// residue planes [batch][N][out_rows][kpad] of the integer images (beta bits) of one operand,
// side and layout as the slice split; exponents as the slice split
void launch_residue_split(const SplitParams& p, const Oz2Tables& T, int max_rows, int batch, cudaStream_t st);
struct CrtParams {
  const int* R;                  // [batch][N][m][ldr] exact integer products (stacked columns)
  long long ldr, plane;          // row pitch (>= 2n) and plane size of R
  const int* e; const int* f; long long e_stride, f_stride;
  int m, n, batch, beta;
  double2* C; int ldc; long long cstride;   // problem z output C + z cstride
  double ar, ai, br, bi;
  int mode;                      // EPI_STORE / EPI_LU / EPI_GENERAL
};
void launch_crt(const CrtParams& p, const Oz2Tables& T, cudaStream_t st);
// one launch for operand a (rows_a rows) and, when b is given, operand b as well; kmax: the
// largest K of the problems (selects the kernel instance)
void launch_split(const SplitParams& a, int rows_a, const SplitParams* b, int rows_b, int kmax, int batch,
                  cudaStream_t st);

// ---- slice_gemm.cu: tcgen05 slice-pair GEMM + exact reconstruction
constexpr int MAX_PAIRS = 136;
// EPI_IMINUS: C = I - RN(Z) without reading C (diagonal where the output row equals the column)
// EPI_RESIDUES: add every group's exact integer value to the int32 buffer `resid` (Ozaki-II)
enum EpiMode : int { EPI_STORE = 0, EPI_LU = 1, EPI_GENERAL = 2, EPI_GROUPS = 3, EPI_IMINUS = 4, EPI_RESIDUES = 5 };
struct GemmParams {
  int S;
  int npairs;
  int ngroups;            // G = g_max - 1
  int kblocks;            // K' / 16 rounded up (uniform over the batch)
  int chunk_kb;           // K-blocks per exactness chunk
  int nstage;
  int mode;
  int base_exp;           // -2B + 8 (2S - g_max)
  int magic;              // 1: every accumulator stays below 2^22 (FP32 add-and-reinterpret conversion)
  int magic_mask;         // bit g: the accumulators of group g stay within 2^22 (same conversion)
  int fit64;              // 1: every exact output sum fits in 64 bits (G <= 5, all chunks)
  int ntx, nty, batch;    // tile grid (set by the launcher): column tiles, row tiles, problems
  int fullset;            // 1: all S x S pairs, 0: triangular s + t <= S + 1
  // skip box: outputs with row < skm and complex column < skn are neither computed (whole
  // tiles) nor written (per element); per problem (skm, skn) or single values (skm1, skn1)
  const int* skm; const int* skn; int skm1, skn1;
  // smallest skip box over the problems (host hint, 0 = none) and the resulting number of
  // tiles enumerated per problem (set by the launcher): only tiles not wholly inside a box
  int box_m, box_n, tpp;
  double ar, ai, br, bi;  // alpha, beta
  const int* m;           // per problem rows of C
  const int* n;           // per problem complex columns of C
  double2* const* C;      // per problem output pointer
  const int* ldc;
  const int* e;           // exponents of rows  [batch][e_stride]
  const int* f;           // exponents of cols  [batch][f_stride]
  long long e_stride, f_stride;
  long long* groups;      // EPI_GROUPS: [G][m][2n] int64 of problem 0 (zeroed by the caller)
  int* status;
  // single-problem values, used when m == nullptr (no device tables needed)
  int m1, n1; double2* C1; int ldc1;
  // row-block scatter (crow != nullptr): row r of problem z is row z crow_b + r % crow_b of
  // the output crow[r / crow_b], whose order and leading dimension are crow_n[r / crow_b]
  // (or ldc1 for every output when crow_n is null); rows past that order are not written
  double2* const* crow; int crow_b; const int* crow_n;
  // crow_perm (optional): row block a of the operand plane belongs to output crow[crow_perm[a]]
  const int* crow_perm;
  // remap (optional, with p.m / p.n tables): problem z reads operand plane remap[z].x (left
  // and right operands, row and column exponents) from plane row remap[z].y on, so that
  // several problems share one split; with crow, its output rows follow that plane row
  const int2* remap;
  // EPI_RESIDUES: group g of problem z, row r, stacked column c at resid[((z G + g) m1 + r) ldres + c]
  int* resid; long long ldres;
  int diag_pairs;                // 1: the pair list is not the tri/full set (runtime issue)
  // test hook of the bounded waits (> 0): before any copy or MMA, every CTA waits on a barrier
  // that no thread arrives at with this budget of SM cycles, gives up and exits
  long long stall_cycles;
  // batched problems of different sizes: exclusive prefix sums of every problem's own tile count
  // ([batch + 1] ints on the device, written by launch_tile_prefix before the GEMM); nullptr:
  // every problem enumerates the tile grid of the largest one (uniform batches, single problems)
  const int* tile_prefix;
  // split K (single problems with fewer tiles than SMs): ksplit > 1 work units per tile, unit
  // u covering tile u / ksplit and exactness chunks [c0, c1) of its K; each unit writes the exact
  // 64-bit halves (H, L) of its partial sums to part[(u % ksplit) m + row][stacked column]
  // (longlong2) and finish_split adds the units and rounds once
  int ksplit;
  longlong2* part;
  uint8_t ps[MAX_PAIRS], pt[MAX_PAIRS], pg[MAX_PAIRS], pfirst[MAX_PAIRS];
};
void launch_slice_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmParams& p, int BN,
                       int max_m, int max_n, int batch, cudaStream_t st);
// the tile prefix sums of a batched GEMM (p.m, p.n and the skip-box tables) into out[0..batch]
void launch_tile_prefix(const GemmParams& p, int BN, int batch, int* out, cudaStream_t st);
// the split-K units' partial sums of a single problem added, rounded once and combined with C
// (the modes of the slice GEMM's epilogue: store, LU, general)
void launch_finish_split(const GemmParams& p, cudaStream_t st);
int gpu_sm_count();
size_t gemm_smem_bytes(int S, int BN, int nstage);

// ---- dmma.cu: binary64 DMMA ZGEMM
struct DmmaParams {
  int m, n, k;
  int transa, conja, transb, conjb;
  const double2* A; long long lda;
  const double2* B; long long ldb;
  double2* C; long long ldc;
  double ar, ai, br, bi;
  // batched form (tm != nullptr): problem z = blockIdx.z takes its sizes, pointers and leading
  // dimensions from these device tables; m, n above are then the largest sizes (grid extent)
  int batch;
  const int *tm, *tn, *tk;
  const double2* const* tA; const int* tlda;
  const double2* const* tB; const int* tldb;
  double2* const* tC; const int* tldc;
};
void launch_dmma(const DmmaParams& p, cudaStream_t st);
// out[z] = base + z * stride and ld[z] = ldv for z < n (pointer tables of per-problem scratch)
void launch_strided_ptrs(double2** out, int* ld, double2* base, long long stride, int ldv, int n, cudaStream_t st);

// ---- lu.cu: Gauss-Jordan solves, M build, scaling
struct GjParams {
  const double2* const* D;  // per problem: nb x nb block, column major
  const int* ldd;
  const int* nb;            // per problem size (0 = skip)
  const double2* const* R;  // per problem right-hand side (nb x nrhs col major) or nullptr = identity
  const int* ldr;
  double2* const* X;        // per problem output nb x nrhs
  const int* ldx;
  int nrhs;                 // columns of R (== nb when R is the identity)
  // single-problem values, used when D == nullptr
  const double2* D1; int ldd1, nb1; const double2* R1; int ldr1; double2* X1; int ldx1;
  int* status;
};
void launch_gj(const GjParams& p, int max_nb, int max_nrhs, int batch, cudaStream_t st);
// X = D^-1 in place (Gauss-Jordan with partial pivoting), blocks of order <= GJINV_MAX; R, nrhs
// unused
constexpr int GJINV_MAX = OZK_NB_MAX;
void launch_gjinv(const GjParams& p, int max_w, int batch, cudaStream_t st);
// P D = L U in place (w <= GJINV_MAX) with the row interchanges applied to the row strip Rs
// (w x ncols, leading dimension ldr) as well
void launch_lu_panel(double2* D, long long ldd, int w, double2* Rs, long long ldr, int ncols, int* status,
                     cudaStream_t st);
// X = inverse of the r x r triangular block T (upper or lower; unit: ones on the diagonal)
constexpr int TRI_INV_MAX = 32;
void launch_tri_inv(const double2* T, long long ldt, int r, int upper, int unit, double2* X, long long ldx, int* status,
                    cudaStream_t st);
void launch_build_m(int n, int b, const double2* t, const double2* G, double2* M, cudaStream_t st);
void launch_build_m_batched(const int* L, int b, const double2* const* t, const double2* const* G, double2* const* M,
                            int nmax, int batch, cudaStream_t st);
void launch_scale(int m, int n, double2* C, long long ldc, double br, double bi, cudaStream_t st);
// Lt (device, per atom block counts) may be null: every atom has L blocks
// perm (optional): position a of the stack holds atom perm[a]
void launch_stack_t(const double2* const* t, const int* Lt, const int* perm, int natoms, int L, int b, double2* out,
                    cudaStream_t st);
void launch_fill_test(double2* const* M, const int* n, int nsolves, int b, double2* t0, cudaStream_t st);
// dst[0..2] = a, b, c (device pointer table of a one-solve call of the batched solver)
void launch_set_ptrs(void** dst, void* a, void* b, void* c, cudaStream_t st);
void launch_contour_trace(const double2* const* tau, int nsolves, int b, const double2* w, double2* tr, double2* out,
                          cudaStream_t st);

// Per-step tables of the batched tau_00 driver, filled on the device for one leaf of one panel.
struct KkrStep {
  // pivot block inverse of the leaf (or, at the end, the S_00^-1 t_0 solve)
  const double2** D; int* ldd; int* nbv; double2** X; int* ldx;
  // GEMM 1: L = M[0:a, a:hi] D^-1 in place
  const double2** A1; int* lda1; const double2** B1; int* ldb1; double2** C1; int* ldc1; int* m1; int* n1; int* k1;
  // GEMM 2: the leaf's frame update M[0:a, 0:a] -= L M[a:hi, 0:a] outside the box [0, p) x [0, p)
  const double2** A2; int* lda2; const double2** B2; int* ldb2; double2** C2; int* ldc2; int* m2; int* n2; int* k2;
  int* skm2; int* skn2;
  // GEMM 3 (last leaf of a panel): the panel's deferred update M[0:p, 0:p] -= M[0:p, p:q] M[p:q, 0:p]
  const double2** A3; int* lda3; const double2** B3; int* ldb3; double2** C3; int* ldc3; int* m3; int* n3; int* k3;
};
// Panel `panel` of solve i: q = n_i - panel W, p = max(q - W, b); its leaf `leaf` is
// [max(hi - w, p), hi) with hi = q - leaf w (absent when hi <= p); D^-1 goes to dinv + i w w
// (pitch w).  The leaf's frame update is empty when the leaf starts at p; GEMM 3 is filled for
// leaf == nleaves - 1 only.  panel < 0: the final S_00^-1 t_0 solve (D = the centre block).
// Solves with nothing left to eliminate get empty problems.
void launch_kkr_step(int panel, int leaf, int nleaves, int nsolves, const int* n, double2* const* M, int b, int W,
                     int w, double2* dinv, const KkrStep& t, cudaStream_t st);

// ---- selector.cu: slice-count selector (features, probes, residual check, perceptron)
constexpr int SEL_NF = OZK_SEL_FEATURES, SEL_NH = 64, SEL_NO = OZK_SEL_OUTPUTS;
constexpr int SEL_SMIN = OZK_SEL_SMIN, SEL_SMAX = OZK_SEL_SMAX, SEL_PROBES = 4;
constexpr int SEL_NPARAMS = OZK_SEL_NPARAMS;
static_assert(SEL_NPARAMS == SEL_NH * SEL_NF + SEL_NH + SEL_NH * SEL_NH + SEL_NH + SEL_NO * SEL_NH + SEL_NO,
              "selector parameter count");
// per-vector arrays; cr: the crest log2 |v|_max + log2 sqrt(2 len) - log2 ||v|| of a nonzero vector
struct SelVecStats { double* r; int* e; double* sh; int* z; double* cr; };
struct SelBases { uint64_t b[2 * SEL_PROBES]; };                 // SplitMix64 stream bases
struct SelAux { int S; int E; double z2; double resid; double diff; float pred[SEL_NO]; };
uint64_t sm_base_host(uint64_t seed, uint64_t stream);
void launch_probe(double2* X, int n, const SelBases& b, cudaStream_t st);
void launch_vec_stats(const double2* M, long long ld, int count, int len, bool contiguous, const SelVecStats& out,
                      cudaStream_t st);
void launch_max_exp(const SelVecStats& a, int ma, const SelVecStats& b, int nb, int* ex, cudaStream_t st);
// Y = (2^-E op(M)) X in double-double (Yh + Yl, ld rows; Xl may be null), compensated sums.
// op: 0 = rows of M (strided; uses `part`, gemv_chunks(len) x SEL_PROBES x rows x 2 double2),
// 1 = columns of M, 2 = conjugated columns of M
int gemv_chunks(int len);
// plain: binary64 sums inside each chunk of the row-strided form (the chunk partials still
// added in double-double)
void launch_gemv(const double2* M, long long ld, int rows, int len, int op, const double2* Xh, const double2* Xl,
                 int ldx, double2* Yh, double2* Yl, double2* part, const int* ex, int eidx, cudaStream_t st,
                 bool plain = false);
void launch_selector_features(const SelVecStats& a, int m, const SelVecStats& b, int n, int k, const double2* X,
                              const double2* zs, const int* ex, float* f, SelAux* aux, cudaStream_t st);
// rpart: scratch of two doubles per block, min(256, ceil(4 m / 256)) blocks (the partials)
void launch_residual(const double2* Wh, const double2* Wl, const double2* zh, const double2* zl, int m, SelAux* aux,
                     double* rpart, cudaStream_t st);
void launch_rel_diff(int m, int n, const double2* X, long long ldx, const double2* Y, long long ldy, double* part,
                     double* out, cudaStream_t st);
void launch_axpby(int m, int n, const double2* D, long long ldd, double2* C, long long ldc, double ar, double ai,
                  double br, double bi, cudaStream_t st);
void launch_mlp_forward(const float* P, const float* X, int N, float* Z1, float* Z2, float* Y, cudaStream_t st);
void launch_mlp_train(float* P, float* gbuf, float* m, float* v, int t, float lr, const float* X, const float* T,
                      int N, float* Z1, float* Z2, float* Y, float* dY, float* dZ2, float* dZ1, double* loss,
                      cudaStream_t st);
void launch_mlp_grad_only(const float* P, float* gbuf, const float* X, const float* T, int N, float* Z1, float* Z2,
                          float* Y, float* dY, float* dZ2, float* dZ1, cudaStream_t st);
void launch_choose(const float* Y, float lim, SelAux* aux, cudaStream_t st);
// Record of the deferred residual checks of the S = 0 GEMMs of one solve: failed = 1 once a
// residual estimate exceeds its bound (or is not finite), the GEMMs counted per S = 3..10, the
// largest residual estimate and the predictions of the last GEMM.
struct SelDefer { int failed; int count[SEL_NO]; double max_resid; float pred[SEL_NO]; };
void launch_defer_check(const SelAux* aux, int S, bool with_pred, double pass, SelDefer* rec, cudaStream_t st);
// *dst = log10(*rel) floored at -17 (selector training targets)
void launch_log_err(const double* rel, float* dst, cudaStream_t st);

}  // namespace ozk
