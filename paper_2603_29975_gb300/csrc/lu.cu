// KKR kernels around the emulated GEMMs (paper Sec. 3.2: LU-based inversion of the
// multiple scattering matrix M = I - t G, whose central block gives tau_00):
//   * gj_solve_kernel  : Gauss-Jordan elimination with partial pivoting on [D | R] for a
//                        batch of small blocks (D up to 64 x 64): R = I gives D^-1 (the
//                        pivot-block inverse of the block LU), R = t_0 gives S_00^-1 t_0.
//   * gjinv_kernel     : in-place Gauss-Jordan inversion with partial pivoting of pivot blocks
//                        up to 112 x 112 (the panel's D^-1 of the block LU).
//   * build_m_kernel   : M = I - blockdiag(t) G.
//   * scale_kernel     : C = beta C (the k == 0 / alpha == 0 case of the GEMM API).
// These are the only places with O(n b^2) / O(n^2 b) binary64 arithmetic of the solve.
#include <algorithm>

#include "ozk_params.cuh"

namespace ozk {

constexpr int GJ_THREADS = 256;



__global__ void __launch_bounds__(GJ_THREADS)
gj_solve_kernel(const GjParams p) {
  extern __shared__ double2 A[];            // [nb][w] row-major, w = nb + nrhs
  __shared__ double2 fcol[64];
  __shared__ int s_piv;
  __shared__ double s_pval;
  const int z = blockIdx.x;
  const bool single = p.D == nullptr;
  const int nb = single ? p.nb1 : p.nb[z];
  if (nb <= 0) return;
  const double2* D = single ? p.D1 : p.D[z];
  const long long ldd = single ? p.ldd1 : p.ldd[z];
  const double2* R = single ? p.R1 : (p.R ? p.R[z] : nullptr);
  const long long ldr = single ? p.ldr1 : (p.R ? p.ldr[z] : 0);
  double2* X = single ? p.X1 : p.X[z];
  const long long ldx = single ? p.ldx1 : p.ldx[z];
  const int nrhs = R ? p.nrhs : nb;
  const int w = nb + nrhs;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < nb * w; idx += GJ_THREADS) {
    const int r = idx % nb, c = idx / nb;
    double2 v;
    if (c < nb) v = D[r + c * ldd];
    else if (R) v = R[r + (c - nb) * ldr];
    else v = make_double2((c - nb) == r ? 1.0 : 0.0, 0.0);
    A[r * w + c] = v;
  }
  __syncthreads();
  bool singular = false;
  for (int pc = 0; pc < nb; ++pc) {
    if (tid < 32) {
      double best = -1.0;
      int bi = pc;
      for (int r = pc + tid; r < nb; r += 32) {
        const double2 v = A[r * w + pc];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) { s_piv = bi; s_pval = best; }
    }
    __syncthreads();
    const int piv = s_piv;
    if (s_pval == 0.0) { singular = true; break; }
    if (piv != pc)
      for (int c = tid; c < w; c += GJ_THREADS) {
        const double2 t = A[pc * w + c];
        A[pc * w + c] = A[piv * w + c];
        A[piv * w + c] = t;
      }
    __syncthreads();
    const double2 pv = A[pc * w + pc];
    const double den = pv.x * pv.x + pv.y * pv.y;
    const double ir = pv.x / den, ii = -pv.y / den;
    __syncthreads();
    for (int c = pc + tid; c < w; c += GJ_THREADS) {
      const double2 x = A[pc * w + c];
      A[pc * w + c] = make_double2(x.x * ir - x.y * ii, x.x * ii + x.y * ir);
    }
    for (int r = tid; r < nb; r += GJ_THREADS) fcol[r] = (r == pc) ? make_double2(0.0, 0.0) : A[r * w + pc];
    __syncthreads();
    const int wc = w - pc;
    for (int idx = tid; idx < nb * wc; idx += GJ_THREADS) {
      const int r = idx / wc, c = pc + idx % wc;
      const double2 f = fcol[r];
      if (f.x != 0.0 || f.y != 0.0) {
        const double2 x = A[pc * w + c];
        double2 y = A[r * w + c];
        y.x -= f.x * x.x - f.y * x.y;
        y.y -= f.x * x.y + f.y * x.x;
        A[r * w + c] = y;
      }
    }
    __syncthreads();
  }
  if (singular) {
    if (tid == 0) flag_error(p.status, OZK_ERR_SINGULAR);
  }
  for (int idx = tid; idx < nb * nrhs; idx += GJ_THREADS) {
    const int r = idx % nb, c = idx / nb;
    X[r + c * ldx] = singular ? make_double2(0.0, 0.0) : A[r * w + nb + c];
  }
}

// Small blocks (nb <= 16, nb + nrhs <= 32): 128 threads per problem, so the binary64 work of
// every elimination step is spread over all four SM sub-partitions (binary64 issue is the
// scarce resource on this GPU); the pivot search and the single complex reciprocal of a step
// are done by one warp / one thread.
constexpr int GJ16_THREADS = 128;

__global__ void __launch_bounds__(GJ16_THREADS)
gj16_kernel(const GjParams p) {
  __shared__ double2 A[16][33];
  __shared__ double2 fcol[16];
  __shared__ int s_piv, s_sing;
  __shared__ double s_ir, s_ii;
  const int z = blockIdx.x;
  const int tid = threadIdx.x;
  const bool single = p.D == nullptr;
  const int nb = single ? p.nb1 : p.nb[z];
  if (nb <= 0) return;
  const double2* D = single ? p.D1 : p.D[z];
  const long long ldd = single ? p.ldd1 : p.ldd[z];
  const double2* R = single ? p.R1 : (p.R ? p.R[z] : nullptr);
  const long long ldr = single ? p.ldr1 : (p.R ? p.ldr[z] : 0);
  double2* X = single ? p.X1 : p.X[z];
  const long long ldx = single ? p.ldx1 : p.ldx[z];
  const int nrhs = R ? p.nrhs : nb;
  const int w = nb + nrhs;
  for (int idx = tid; idx < nb * w; idx += GJ16_THREADS) {
    const int r = idx % nb, c = idx / nb;
    double2 v;
    if (c < nb) v = D[r + c * ldd];
    else if (R) v = R[r + (c - nb) * ldr];
    else v = make_double2((c - nb) == r ? 1.0 : 0.0, 0.0);
    A[r][c] = v;
  }
  if (tid == 0) s_sing = 0;
  __syncthreads();
  for (int pc = 0; pc < nb; ++pc) {
    if (tid < 32) {
      // partial pivoting: first row of largest |.|^2 in column pc (lane = row)
      double best = -1.0;
      int bi = pc;
      if (tid >= pc && tid < nb) {
        const double2 v = A[tid][pc];
        best = v.x * v.x + v.y * v.y;
        bi = tid;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        if (best <= 0.0) {
          s_sing = 1;
        } else {
          const double2 v = A[bi][pc];
          const double inv = 1.0 / best;                 // the one division of the step
          s_ir = v.x * inv;
          s_ii = -v.y * inv;
        }
      }
    }
    __syncthreads();
    if (s_sing) break;
    const int piv = s_piv;
    if (tid < w) {                                       // swap rows pc, piv and scale row pc
      const double2 t = A[piv][tid];
      if (piv != pc) A[piv][tid] = A[pc][tid];
      A[pc][tid] = make_double2(t.x * s_ir - t.y * s_ii, t.x * s_ii + t.y * s_ir);
    }
    __syncthreads();
    if (tid < nb) fcol[tid] = (tid == pc) ? make_double2(0.0, 0.0) : A[tid][pc];
    __syncthreads();
    const int wc = w - pc;                               // columns pc .. w-1
    for (int idx = tid; idx < nb * wc; idx += GJ16_THREADS) {
      const int r = idx % nb, c = pc + idx / nb;
      if (r == pc) continue;
      if (c == pc) { A[r][c] = make_double2(0.0, 0.0); continue; }
      const double2 f = fcol[r];
      const double2 x = A[pc][c];
      double2 y = A[r][c];
      y.x -= f.x * x.x - f.y * x.y;
      y.y -= f.x * x.y + f.y * x.x;
      A[r][c] = y;
    }
    __syncthreads();
  }
  const bool singular = s_sing != 0;
  if (singular && tid == 0) flag_error(p.status, OZK_ERR_SINGULAR);
  for (int idx = tid; idx < nb * nrhs; idx += GJ16_THREADS) {
    const int r = idx % nb, c = idx / nb;
    X[r + c * ldx] = singular ? make_double2(0.0, 0.0) : A[r][nb + c];
  }
}

// In-place Gauss-Jordan inversion with partial pivoting: X = D^-1 for a batch of pivot blocks
// of order w <= GJINV_MAX (the nb x nb diagonal block of a block-LU panel).  Step k swaps row k
// with the row of largest |.|^2 in column k (at or below k), scales the row by the pivot's
// reciprocal, eliminates column k from every other row and stores the k-th column of the
// inverse in its place; after the last step the row interchanges are undone as column
// interchanges in reverse order.  w^2 complex of shared memory (the [D | I] form of
// gj_solve_kernel needs twice that) and w^3 complex multiply-adds per block.
constexpr int GJINV_THREADS = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(GJINV_THREADS)
gjinv_kernel(const GjParams p, int skip_lo, int skip_hi) {
  extern __shared__ double2 A[];            // [w][w] column major
  __shared__ double2 colk[GJINV_MAX];
  __shared__ int perm[GJINV_MAX];
  __shared__ int src[GJINV_MAX];
  __shared__ int s_piv, s_sing;
  __shared__ double2 s_pinv;
  const int z = blockIdx.x;
  const bool single = p.D == nullptr;
  const int w = single ? p.nb1 : p.nb[z];
  if (w <= 0 || (w > skip_lo && w <= skip_hi)) return;  // those blocks: gjinv_reg_kernel
  const double2* D = single ? p.D1 : p.D[z];
  const long long ldd = single ? p.ldd1 : p.ldd[z];
  double2* X = single ? p.X1 : p.X[z];
  const long long ldx = single ? p.ldx1 : p.ldx[z];
  const int tid = threadIdx.x;
  const int ww = w * w;
  for (int idx = tid; idx < ww; idx += GJINV_THREADS) {
    const int j = idx / w, i = idx - j * w;
    A[idx] = D[i + j * ldd];
  }
  if (tid == 0) s_sing = 0;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    if (tid < 32) {
      // partial pivoting: first row of largest |.|^2 in column k at or below row k
      double best = -1.0;
      int bi = k;
      for (int r = k + tid; r < w; r += 32) {
        const double2 v = A[r + k * w];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        perm[k] = bi;
        if (best <= 0.0) {
          s_sing = 1;
        } else {
          const double2 v = A[bi + k * w];
          const double inv = 1.0 / best;               // the one division of the step
          s_pinv = make_double2(v.x * inv, -v.y * inv);
        }
      }
    }
    __syncthreads();
    if (s_sing) break;
    const int piv = s_piv;
    const double2 pinv = s_pinv;
    // rows k and piv exchanged outside column k, the new row k scaled; column k as it reads
    // after the exchange (zero in the pivot row) kept aside -- no thread writes it here
    for (int j = tid; j < w; j += GJINV_THREADS) {
      if (j == k) continue;
      const double2 a = A[k + j * w], b = A[piv + j * w];
      if (piv != k) A[piv + j * w] = a;
      A[k + j * w] = cmul(b, pinv);
    }
    for (int i = tid; i < w; i += GJINV_THREADS)
      colk[i] = (i == k) ? make_double2(0.0, 0.0) : A[(i == piv ? k : i) + k * w];
    __syncthreads();
    for (int idx = tid; idx < ww; idx += GJINV_THREADS) {
      const int j = idx / w, i = idx - j * w;
      if (j == k) {
        const double2 c = cmul(colk[i], pinv);
        A[idx] = (i == k) ? pinv : make_double2(-c.x, -c.y);
      } else if (i != k) {
        // y -= f x as four fused multiply-adds (binary64 issue is the scarce resource)
        const double2 f = colk[i];
        const double2 x = A[k + j * w];
        double2 y = A[idx];
        y.x = fma(-f.x, x.x, y.x);
        y.x = fma(f.y, x.y, y.x);
        y.y = fma(-f.x, x.y, y.y);
        y.y = fma(-f.y, x.x, y.y);
        A[idx] = y;
      }
    }
    __syncthreads();
  }
  const bool singular = s_sing != 0;
  if (tid == 0) {
    if (singular) flag_error(p.status, OZK_ERR_SINGULAR);
    for (int j = 0; j < w; ++j) src[j] = j;
    if (!singular)
      for (int k = w - 1; k >= 0; --k) {
        const int r = perm[k];
        if (r != k) { const int t = src[k]; src[k] = src[r]; src[r] = t; }
      }
  }
  __syncthreads();
  for (int idx = tid; idx < ww; idx += GJINV_THREADS) {
    const int j = idx / w, i = idx - j * w;
    X[i + j * ldx] = singular ? make_double2(0.0, 0.0) : A[i + src[j] * w];
  }
}

// The same Gauss-Jordan inversion for blocks of order w <= 64 with the block held in
// registers: thread t keeps column j = t mod 64, rows rb + 4c (rb = t / 64, c = 0..15), 16
// complex values; 256 threads, two warps per SM sub-partition (one warp per sub-partition
// leaves the binary64 multiply-add chains exposed: 413 against 350 us per 64 x 64 block).
// Step k: the owner threads of column k publish it, one warp picks the pivot (the row of
// largest |.|^2 at or below k, the first on ties; the keys are compared as the integer images
// of the non-negative binary64 |.|^2, which orders them exactly, a NaN never wins), the owners
// of rows piv and k publish the scaled pivot row and the old row k, and every thread
// eliminates column k from its 16 rows with the same four fused multiply-adds per complex
// entry as above.  Column k of the inverse is formed by the same multiply-adds from zero
// (y = 0 - f * pinv).  Rows and columns at or beyond w are zero padding and never written out.
// w^3 complex multiply-adds per block, as in gjinv_kernel; 350 against 423 us per 64 x 64
// block on one SM.  Its 128 registers a thread fill half of an SM's register file, so two
// such CTAs on one SM leave no room for the side stream's split CTAs that run beside the
// shared-memory kernel: it serves launches of at most one block per SM.  Rows at or beyond w
// are skipped, but a warp spans 32 columns whatever w is, so narrower blocks (w = 48: 3/4 of
// the lanes busy) stay with the shared-memory kernel.
constexpr int GJR_THREADS = 256;
constexpr int GJR_W = 64;
constexpr int GJR_MIN_W = 56;                   // narrower blocks stay with gjinv_kernel
constexpr int GJR_RG = GJR_THREADS / GJR_W;     // row groups
constexpr int GJR_RPT = GJR_W / GJR_RG;         // rows per thread

__device__ __forceinline__ double2 pick_row(const double2 (&a)[GJR_RPT], int c) {
  double2 v = a[0];
#pragma unroll
  for (int q = 1; q < GJR_RPT; ++q)
    if (q == c) v = a[q];
  return v;
}

__global__ void __launch_bounds__(GJR_THREADS, 2)
gjinv_reg_kernel(const GjParams p) {
  __shared__ double2 colbuf[GJR_W];        // column k before the exchange
  __shared__ double2 colk[GJR_W];          // column k after the exchange, pivot row zeroed
  __shared__ double2 newk[GJR_W];          // the pivot row scaled by 1 / pivot (the new row k)
  __shared__ double2 oldk[GJR_W];          // row k before the exchange (the new row piv)
  __shared__ int perm[GJR_W], src[GJR_W], dst[GJR_W];
  __shared__ int s_piv, s_sing;
  __shared__ double2 s_pinv;
  const int z = blockIdx.x;
  const bool single = p.D == nullptr;
  const int w = single ? p.nb1 : p.nb[z];
  if (w <= GJR_MIN_W || w > GJR_W) return;             // gjinv_kernel's blocks
  const double2* D = single ? p.D1 : p.D[z];
  const long long ldd = single ? p.ldd1 : p.ldd[z];
  double2* X = single ? p.X1 : p.X[z];
  const long long ldx = single ? p.ldx1 : p.ldx[z];
  const int tid = threadIdx.x;
  const int j = tid & (GJR_W - 1), rb = tid / GJR_W;
  double2 a[GJR_RPT];
#pragma unroll
  for (int c = 0; c < GJR_RPT; ++c) {
    const int i = rb + GJR_RG * c;
    a[c] = (i < w && j < w) ? D[i + j * ldd] : make_double2(0.0, 0.0);
  }
  if (tid == 0) s_sing = 0;
  if (j == 0) {
#pragma unroll
    for (int c = 0; c < GJR_RPT; ++c) colbuf[rb + GJR_RG * c] = a[c];
  }
  for (int k = 0; k < w; ++k) {
    __syncthreads();                                    // column k is in colbuf
    if (tid < 32) {
      long long best = -1;                              // no candidate yet
      int bi = k;
      for (int r = k + tid; r < w; r += 32) {
        const double2 v = colbuf[r];
        long long key = __double_as_longlong(v.x * v.x + v.y * v.y);
        if (key > 0x7FF0000000000000LL) key = -1;         // NaN
        if (key > best) { best = key; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        perm[k] = bi;
        if (best <= 0) {
          s_sing = 1;
        } else {
          const double2 v = colbuf[bi];
          const double inv = 1.0 / __longlong_as_double(best);   // the one division of the step
          s_pinv = make_double2(v.x * inv, -v.y * inv);
        }
      }
    }
    __syncthreads();
    if (s_sing) break;
    const int piv = s_piv;
    const double2 pinv = s_pinv;
    if (rb == piv % GJR_RG) newk[j] = cmul(pick_row(a, piv / GJR_RG), pinv);
    if (rb == k % GJR_RG) oldk[j] = pick_row(a, k / GJR_RG);
    if (tid < GJR_W)
      colk[tid] = (tid == k || tid >= w) ? make_double2(0.0, 0.0) : colbuf[tid == piv ? k : tid];
    __syncthreads();
    const bool colK = j == k;
    const double2 x = colK ? pinv : newk[j];
    const double2 ok = oldk[j];
#pragma unroll
    for (int c = 0; c < GJR_RPT; ++c) {
      const int i = rb + GJR_RG * c;
      if (i >= w || j >= w) continue;                   // padding (i is uniform across a warp)
      const double2 f = colk[i];
      double2 y = colK ? make_double2(0.0, 0.0) : (i == piv ? ok : a[c]);
      y.x = fma(-f.x, x.x, y.x);
      y.x = fma(f.y, x.y, y.x);
      y.y = fma(-f.x, x.y, y.y);
      y.y = fma(-f.y, x.x, y.y);
      a[c] = (i == k) ? x : y;
    }
    if (j == k + 1) {                                   // publish the next step's column
#pragma unroll
      for (int c = 0; c < GJR_RPT; ++c) colbuf[rb + GJR_RG * c] = a[c];
    }
  }
  __syncthreads();
  const bool singular = s_sing != 0;
  if (tid == 0) {
    if (singular) flag_error(p.status, OZK_ERR_SINGULAR);
    for (int q = 0; q < w; ++q) src[q] = q;
    if (!singular)
      for (int q = w - 1; q >= 0; --q) {
        const int r = perm[q];
        if (r != q) { const int t = src[q]; src[q] = src[r]; src[r] = t; }
      }
    for (int q = 0; q < w; ++q) dst[src[q]] = q;        // column j of the block is column dst[j] of X
  }
  __syncthreads();
  if (j < w) {
    double2* xo = X + static_cast<long long>(dst[j]) * ldx;
#pragma unroll
    for (int c = 0; c < GJR_RPT; ++c) {
      const int i = rb + GJR_RG * c;
      if (i < w) xo[i] = singular ? make_double2(0.0, 0.0) : a[c];
    }
  }
}

// In-place LU factorisation with partial pivoting of a w x w pivot block (w <= GJINV_MAX,
// binary64): P D = L U with L unit lower triangular (its multipliers stored below the
// diagonal) and U upper triangular, written back over D; every row interchange of step k is
// applied to the whole block row, and afterwards -- in the same order -- to the rows of the
// panel's row strip Rs (w rows, ncols columns, leading dimension ldr), so that the trailing
// update can use the interchanged strip directly.  w^3 / 3 complex multiply-adds.
__global__ void __launch_bounds__(GJINV_THREADS)
lu_panel_kernel(double2* D, long long ldd, int w, double2* Rs, long long ldr, int ncols, int* status) {
  extern __shared__ double2 A[];            // [w][w] column major
  __shared__ int perm[GJINV_MAX];
  __shared__ int s_piv, s_sing;
  __shared__ double2 s_pinv;
  const int tid = threadIdx.x;
  const int ww = w * w;
  for (int idx = tid; idx < ww; idx += GJINV_THREADS) {
    const int j = idx / w, i = idx - j * w;
    A[idx] = D[i + j * ldd];
  }
  if (tid == 0) s_sing = 0;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + tid; r < w; r += 32) {
        const double2 v = A[r + k * w];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        perm[k] = bi;
        if (best <= 0.0) {
          s_sing = 1;
        } else {
          const double2 v = A[bi + k * w];
          const double inv = 1.0 / best;               // the one division of the step
          s_pinv = make_double2(v.x * inv, -v.y * inv);
        }
      }
    }
    __syncthreads();
    if (s_sing) break;
    const int piv = s_piv;
    if (piv != k)
      for (int j = tid; j < w; j += GJINV_THREADS) {
        const double2 t = A[k + j * w];
        A[k + j * w] = A[piv + j * w];
        A[piv + j * w] = t;
      }
    __syncthreads();
    const double2 pinv = s_pinv;
    for (int i = k + 1 + tid; i < w; i += GJINV_THREADS) A[i + k * w] = cmul(A[i + k * w], pinv);
    __syncthreads();
    const int r = w - k - 1;                // trailing block rows / columns k+1 .. w-1
    for (int idx = tid; idx < r * r; idx += GJINV_THREADS) {
      const int jj = idx / r, ii = idx - jj * r;
      const int i = k + 1 + ii, j = k + 1 + jj;
      const double2 l = A[i + k * w], u = A[k + j * w];
      double2 y = A[i + j * w];
      y.x = fma(-l.x, u.x, y.x);
      y.x = fma(l.y, u.y, y.x);
      y.y = fma(-l.x, u.y, y.y);
      y.y = fma(-l.y, u.x, y.y);
      A[i + j * w] = y;
    }
    __syncthreads();
  }
  const bool singular = s_sing != 0;
  if (singular && tid == 0) flag_error(status, OZK_ERR_SINGULAR);
  for (int idx = tid; idx < ww; idx += GJINV_THREADS) {
    const int j = idx / w, i = idx - j * w;
    D[i + j * ldd] = A[idx];
  }
  if (singular) return;
  // the same interchanges, in order, on the row strip
  for (int k = 0; k < w; ++k) {
    const int pk = perm[k];
    if (pk != k)
      for (int j = tid; j < ncols; j += GJINV_THREADS) {
        const double2 t = Rs[k + j * ldr];
        Rs[k + j * ldr] = Rs[pk + j * ldr];
        Rs[pk + j * ldr] = t;
      }
    __syncthreads();
  }
}

void launch_lu_panel(double2* D, long long ldd, int w, double2* Rs, long long ldr, int ncols, int* status,
                     cudaStream_t st) {
  const size_t smem = sizeof(double2) * static_cast<size_t>(w) * w;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(lu_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  lu_panel_kernel<<<1, GJINV_THREADS, smem, st>>>(D, ldd, w, Rs, ldr, ncols, status);
  record_launch();
}

// Inverse of the r x r triangular diagonal block T (leading dimension ldt) into X (leading
// dimension ldx), binary64: upper or lower triangular, with its stored diagonal or (unit) with
// ones there.  The other triangle of T is ignored.  Thread c computes column c by substitution.
// r <= TRI_INV_MAX.
// a / d for a nonzero d; flags a singular block and returns 0 otherwise
__device__ __forceinline__ double2 cdiv_checked(double2 a, double2 d, int* status) {
  const double den = d.x * d.x + d.y * d.y;
  if (den == 0.0) { flag_error(status, OZK_ERR_SINGULAR); return make_double2(0.0, 0.0); }
  return make_double2((a.x * d.x + a.y * d.y) / den, (a.y * d.x - a.x * d.y) / den);
}

__global__ void tri_inv_kernel(const double2* T, long long ldt, int r, int upper, int unit, double2* X, long long ldx,
                               int* status) {
  __shared__ double2 t[TRI_INV_MAX][TRI_INV_MAX + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < r * r; idx += blockDim.x) {
    const int j = idx / r, i = idx - j * r;
    t[i][j] = T[i + j * ldt];
  }
  __syncthreads();
  for (int c = tid; c < r; c += blockDim.x) {
    double2 x[TRI_INV_MAX];
    if (upper) {
      for (int i = r - 1; i >= 0; --i) {
        if (i > c) { x[i] = make_double2(0.0, 0.0); continue; }
        double2 acc = make_double2(i == c ? 1.0 : 0.0, 0.0);
        for (int j = i + 1; j <= c; ++j) {
          const double2 u = t[i][j];
          acc.x -= u.x * x[j].x - u.y * x[j].y;
          acc.y -= u.x * x[j].y + u.y * x[j].x;
        }
        x[i] = unit ? acc : cdiv_checked(acc, t[i][i], status);
      }
    } else {
      for (int i = 0; i < r; ++i) {
        if (i < c) { x[i] = make_double2(0.0, 0.0); continue; }
        double2 acc = make_double2(i == c ? 1.0 : 0.0, 0.0);
        for (int j = c; j < i; ++j) {
          const double2 l = t[i][j];
          acc.x -= l.x * x[j].x - l.y * x[j].y;
          acc.y -= l.x * x[j].y + l.y * x[j].x;
        }
        x[i] = unit ? acc : cdiv_checked(acc, t[i][i], status);
      }
    }
    for (int i = 0; i < r; ++i) X[i + c * ldx] = x[i];
  }
}

void launch_tri_inv(const double2* T, long long ldt, int r, int upper, int unit, double2* X, long long ldx, int* status,
                    cudaStream_t st) {
  tri_inv_kernel<<<1, TRI_INV_MAX, 0, st>>>(T, ldt, r, upper, unit, X, ldx, status);
  record_launch();
}

void launch_gjinv(const GjParams& p, int max_w, int batch, cudaStream_t st) {
  // the register form takes the blocks of order 56 < w <= 64 when every block of the launch
  // has an SM to itself, the shared-memory kernel the others; which form inverts a block
  // depends on its own order and the launch's size only, so a block comes out the same alone
  // and in a small batch
  const bool single = p.D == nullptr;                      // one block, of order max_w
  const bool reg = max_w > GJR_MIN_W && batch <= gpu_sm_count() && (!single || max_w <= GJR_W);
  if (reg) {
    gjinv_reg_kernel<<<batch, GJR_THREADS, 0, st>>>(p);
    record_launch();
    if (single) return;
  }
  const size_t smem = sizeof(double2) * static_cast<size_t>(max_w) * max_w;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(gjinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  gjinv_kernel<<<batch, GJINV_THREADS, smem, st>>>(p, reg ? GJR_MIN_W : 0, reg ? GJR_W : 0);
  record_launch();
}

void launch_gj(const GjParams& p, int max_nb, int max_nrhs, int batch, cudaStream_t st) {
  if (max_nb <= 16 && max_nb + max_nrhs <= 32) {
    gj16_kernel<<<batch, GJ16_THREADS, 0, st>>>(p);
  } else {
    const size_t smem = sizeof(double2) * static_cast<size_t>(max_nb) * (max_nb + max_nrhs);
    if (smem > 48 * 1024) cudaFuncSetAttribute(gj_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    gj_solve_kernel<<<batch, GJ_THREADS, smem, st>>>(p);
  }
  record_launch();
}

// M = I - blockdiag(t) G ; t: L blocks b x b (col major, block l at t + l b b); G, M: n x n.
__global__ void build_m_kernel(int n, int b, const double2* __restrict__ t, const double2* __restrict__ G,
                               double2* __restrict__ M) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n) * n) return;
  const int i = static_cast<int>(idx % n), j = static_cast<int>(idx / n);
  const int l = i / b, r = i % b;
  const double2* tl = t + static_cast<long long>(l) * b * b;
  double sr = 0.0, si = 0.0;
  for (int c = 0; c < b; ++c) {
    const double2 a = tl[r + c * b];
    const double2 g = G[(l * b + c) + static_cast<long long>(j) * n];
    sr += a.x * g.x - a.y * g.y;
    si += a.x * g.y + a.y * g.x;
  }
  M[idx] = make_double2((i == j ? 1.0 : 0.0) - sr, -si);
}

void launch_build_m(int n, int b, const double2* t, const double2* G, double2* M, cudaStream_t st) {
  const long long tot = static_cast<long long>(n) * n;
  build_m_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(n, b, t, G, M);
  record_launch();
}

// Batched M_z = I - blockdiag(t_z) G_z over grid.y = problem z (n_z = L_z b).
__global__ void build_m_batched_kernel(const int* __restrict__ L, int b, const double2* const* t,
                                       const double2* const* G, double2* const* M) {
  const int z = blockIdx.y;
  const int n = L[z] * b;
  const double2* __restrict__ tz = t[z];
  const double2* __restrict__ Gz = G[z];
  double2* __restrict__ Mz = M[z];
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < static_cast<long long>(n) * n;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(idx % n), j = static_cast<int>(idx / n);
    const int l = i / b, r = i % b;
    const double2* tl = tz + static_cast<long long>(l) * b * b;
    double sr = 0.0, si = 0.0;
    for (int c = 0; c < b; ++c) {
      const double2 a = tl[r + c * b];
      const double2 g = Gz[(l * b + c) + static_cast<long long>(j) * n];
      sr += a.x * g.x - a.y * g.y;
      si += a.x * g.y + a.y * g.x;
    }
    Mz[idx] = make_double2((i == j ? 1.0 : 0.0) - sr, -si);
  }
}

void launch_build_m_batched(const int* L, int b, const double2* const* t, const double2* const* G, double2* const* M,
                            int nmax, int batch, cudaStream_t st) {
  const long long tot = static_cast<long long>(nmax) * nmax;
  const unsigned gx = static_cast<unsigned>(std::min<long long>((tot + 255) / 256, 4096));
  build_m_batched_kernel<<<dim3(gx, batch), 256, 0, st>>>(L, b, t, G, M);
  record_launch();
}

// Stacked left operands of the shared-G build: problem i is the (natoms b) x b column-major
// matrix whose rows a b .. a b + b - 1 are block i of t_{perm[a]} (t_a: L column-major b x b
// blocks; perm null: the identity).
__global__ void stack_t_kernel(const double2* const* t, const int* Lt, const int* perm, int natoms, int L, int b,
                               double2* out) {
  const long long rows = static_cast<long long>(natoms) * b, per = rows * b;
  const long long tot = per * L;
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(idx / per);
    const long long rem = idx - i * per;
    const int c = static_cast<int>(rem / rows);
    const int ar = static_cast<int>(rem - c * rows);
    const int as = ar / b, r = ar - as * b;
    const int a = perm ? perm[as] : as;
    // block rows past an atom's own LIZ are zero (that atom's rows of the product are not kept)
    out[idx] = (Lt && i >= Lt[a]) ? make_double2(0.0, 0.0)
                                  : t[a][static_cast<long long>(i) * b * b + r + static_cast<long long>(c) * b];
  }
}

// Traces of the b x b blocks tau[i] (column major) and their weighted sum sum_i w_i Tr tau_i:
// one warp per block for the traces, then one block sums the products in order.
__global__ void trace_kernel(const double2* const* tau, int nsolves, int b, double2* tr) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= nsolves) return;
  double re = 0.0, im = 0.0;
  for (int d = lane; d < b; d += 32) {
    const double2 v = tau[i][d + static_cast<long long>(d) * b];
    re += v.x;
    im += v.y;
  }
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) tr[i] = make_double2(re, im);
}

__global__ void weighted_sum_kernel(const double2* tr, const double2* w, int nsolves, double2* out) {
  if (threadIdx.x || blockIdx.x) return;
  double re = 0.0, im = 0.0;
  for (int i = 0; i < nsolves; ++i) {
    re += w[i].x * tr[i].x - w[i].y * tr[i].y;
    im += w[i].x * tr[i].y + w[i].y * tr[i].x;
  }
  *out = make_double2(re, im);
}

void launch_contour_trace(const double2* const* tau, int nsolves, int b, const double2* w, double2* tr, double2* out,
                          cudaStream_t st) {
  trace_kernel<<<(nsolves * 32 + 255) / 256, 256, 0, st>>>(tau, nsolves, b, tr);
  record_launch();
  weighted_sum_kernel<<<1, 32, 0, st>>>(tr, w, nsolves, out);
  record_launch();
}

// Test matrices of the autotuner: M_i = I + off-diagonal entries of magnitude < 0.25 / n_i
// (a fixed integer hash), strictly diagonally dominant so every pivot block is regular; t_0 = I.
__global__ void fill_test_kernel(double2* const* M, const int* n, int b, double2* t0) {
  const int z = blockIdx.y;
  const int ni = n[z];
  const long long tot = static_cast<long long>(ni) * ni;
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(idx % ni), c = static_cast<int>(idx / ni);
    unsigned h = static_cast<unsigned>(r) * 2654435761u ^ static_cast<unsigned>(c) * 40503u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const double u = (static_cast<double>(h & 0xFFFF) / 65536.0 - 0.5) * (0.5 / ni);
    const double w = (static_cast<double>((h >> 16) & 0xFFFF) / 65536.0 - 0.5) * (0.5 / ni);
    M[z][idx] = r == c ? make_double2(1.0, 0.0) : make_double2(u, w);
  }
  if (z == 0 && blockIdx.x == 0)
    for (int i = threadIdx.x; i < b * b; i += blockDim.x) t0[i] = make_double2(i % (b + 1) == 0 ? 1.0 : 0.0, 0.0);
}

__global__ void set_ptrs_kernel(void** dst, void* a, void* b, void* c) {
  if (threadIdx.x == 0) { dst[0] = a; dst[1] = b; dst[2] = c; }
}

void launch_set_ptrs(void** dst, void* a, void* b, void* c, cudaStream_t st) {
  set_ptrs_kernel<<<1, 32, 0, st>>>(dst, a, b, c);
  record_launch();
}

void launch_fill_test(double2* const* M, const int* n, int nsolves, int b, double2* t0, cudaStream_t st) {
  fill_test_kernel<<<dim3(1024, nsolves), 256, 0, st>>>(M, n, b, t0);
  record_launch();
}

void launch_stack_t(const double2* const* t, const int* Lt, const int* perm, int natoms, int L, int b, double2* out,
                    cudaStream_t st) {
  const long long tot = static_cast<long long>(natoms) * b * b * L;
  const unsigned blocks = static_cast<unsigned>(std::min<long long>((tot + 255) / 256, 8192));
  stack_t_kernel<<<blocks, 256, 0, st>>>(t, Lt, perm, natoms, L, b, out);
  record_launch();
}

__global__ void scale_kernel(int m, int n, double2* C, long long ldc, double br, double bi) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(m) * n) return;
  const int i = static_cast<int>(idx % m), j = static_cast<int>(idx / m);
  double2* d = C + i + j * ldc;
  if (br == 0.0 && bi == 0.0) { *d = make_double2(0.0, 0.0); return; }
  const double2 v = *d;
  *d = make_double2(br * v.x - bi * v.y, br * v.y + bi * v.x);
}

void launch_scale(int m, int n, double2* C, long long ldc, double br, double bi, cudaStream_t st) {
  const long long tot = static_cast<long long>(m) * n;
  if (tot == 0) return;
  scale_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(m, n, C, ldc, br, bi);
  record_launch();
}

}  // namespace ozk

namespace ozk {

// Per-solve tables of one step of the batched block LU.  Panel `step` is J = [p, q) with
// q = n - step nb, p = max(q - nb, b), w = q - p: the pivot-block inverse table (D = M[p:q, p:q],
// D^-1 into the solve's nb x nb slot of dinv), GEMM 1 (L = M[0:p, p:q] D^-1, in place) and GEMM 2
// (M[0:p, 0:p] -= L M[p:q, 0:p]); step < 0 the final S_00 solve.  Finished solves get zero
// sizes.
__global__ void kkr_step_kernel(int panel, int leaf, int nleaves, int nsolves, const int* __restrict__ n,
                                double2* const* M, int b, int W, int w, double2* dinv, KkrStep t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsolves) return;
  const int ni = n[i];
  double2* Mi = M[i];
  double2* Di = dinv + static_cast<long long>(i) * w * w;
  // defaults: nothing to do
  t.D[i] = Mi; t.ldd[i] = ni; t.nbv[i] = 0; t.X[i] = Di; t.ldx[i] = w;
  t.A1[i] = Mi; t.lda1[i] = ni; t.B1[i] = Di; t.ldb1[i] = w; t.C1[i] = Mi; t.ldc1[i] = ni;
  t.m1[i] = 0; t.n1[i] = 0; t.k1[i] = b;
  t.A2[i] = Mi; t.lda2[i] = ni; t.B2[i] = Mi; t.ldb2[i] = ni; t.C2[i] = Mi; t.ldc2[i] = ni;
  t.m2[i] = 0; t.n2[i] = 0; t.k2[i] = b; t.skm2[i] = 0; t.skn2[i] = 0;
  t.A3[i] = Mi; t.lda3[i] = ni; t.B3[i] = Mi; t.ldb3[i] = ni; t.C3[i] = Mi; t.ldc3[i] = ni;
  t.m3[i] = 0; t.n3[i] = 0; t.k3[i] = b;
  if (panel < 0) { t.nbv[i] = b; return; }
  const int q = ni - panel * W;
  if (q <= b) return;
  const int p = max(q - W, b);
  if (leaf == nleaves - 1) {                                  // the panel's deferred update
    t.A3[i] = Mi + static_cast<long long>(p) * ni;            // M[0:p, p:q]
    t.B3[i] = Mi + p;                                         // M[p:q, 0:p]
    t.m3[i] = p; t.n3[i] = p; t.k3[i] = q - p;
  }
  const int hi = q - leaf * w;
  if (hi <= p) return;
  const int a = max(hi - w, p), wl = hi - a;
  t.D[i] = Mi + a + static_cast<long long>(a) * ni; t.nbv[i] = wl;
  double2* La = Mi + static_cast<long long>(a) * ni;          // M[0:a, a:hi]
  t.A1[i] = La; t.C1[i] = La; t.m1[i] = a; t.n1[i] = wl; t.k1[i] = wl;
  if (a > p) {                                                // frame of the leaf
    t.A2[i] = La; t.B2[i] = Mi + a; t.m2[i] = a; t.n2[i] = a; t.k2[i] = wl;
    t.skm2[i] = p; t.skn2[i] = p;
  }
}

void launch_kkr_step(int panel, int leaf, int nleaves, int nsolves, const int* n, double2* const* M, int b, int W,
                     int w, double2* dinv, const KkrStep& t, cudaStream_t st) {
  kkr_step_kernel<<<(nsolves + 127) / 128, 128, 0, st>>>(panel, leaf, nleaves, nsolves, n, M, b, W, w, dinv, t);
  record_launch();
}

}  // namespace ozk
