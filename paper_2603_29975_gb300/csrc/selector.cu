// Slice-count selector kernels.
//
// The paper finds that the emulation's accuracy depends on both the slice count and the
// operator and handles it by tuning the precision (Abstract; Sec. 4), arguing for adaptive
// precision (Sec. 5) without a rule for choosing it.  These kernels implement the selector of
// this library:
//   * per-row / per-column operand statistics and a probe product z = op(A) (op(B) X) with
//     counter-based random probe vectors X (SplitMix64: Steele, Lea and Flood, OOPSLA 2014),
//     reduced to 16 features (binary64 arithmetic, float32 features);
//   * a 16 -> 64 -> 64 -> 8 ReLU perceptron predicting log10 relative errors for S = 3..10:
//     forward, backward (mean squared error), per-parameter gradient sums and Adam (Kingma and
//     Ba, ICLR 2015) updates, all float32;
//   * the choice of S and the a-posteriori residual estimate ||2^-E D X - zs|| / ||zs||,
//     whose square has expectation ||D - AB||_F^2 / ||AB||_F^2 for the probe distribution.
// The feature definitions are stated in selector_features_kernel; the parameter layout is
// W1[64][16], b1[64], W2[64][64], b2[64], W3[8][64], b3[8].
#include <math.h>

#include <algorithm>

#include "ozk_params.cuh"

namespace ozk {

// ------------------------------------------------------------------ SplitMix64
__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

uint64_t sm_base_host(uint64_t seed, uint64_t stream) {
  uint64_t z = (seed * 0x100000001B3ull) ^ stream;
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// uniform double in [0, 1) with 53 bits: output number idx of the stream with this base
__device__ __forceinline__ double sm_uniform(uint64_t base, uint64_t idx) {
  return static_cast<double>(sm_mix(base + (idx + 1ull) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}

// X (n x SEL_PROBES, column major): Re of column p from stream 2p, Im from stream 2p + 1,
// (U - 1/2) * sqrt(6), so that every entry has E|x|^2 = 1.
__global__ void probe_kernel(double2* X, int n, SelBases bases) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double c = 2.449489742783178;   // sqrt(6) rounded to binary64
#pragma unroll
  for (int p = 0; p < SEL_PROBES; ++p) {
    double2 v;
    v.x = (sm_uniform(bases.b[2 * p], j) - 0.5) * c;
    v.y = (sm_uniform(bases.b[2 * p + 1], j) - 0.5) * c;
    X[j + static_cast<long long>(p) * n] = v;
  }
}

// ------------------------------------------------------------------ vector statistics
// Vectors are the rows of op(M) (M column major, ld): r = max(|Re|, |Im|), e = frexp exponent
// of r (0 for a zero vector), sh = sum |v 2^-e|^2, z = number of exactly zero entries.
__device__ __forceinline__ int frexp_exp(double r) {
  int e = 0;
  if (r > 0.0) frexp(r, &e);
  return e;
}

// crest of a vector of len complex entries: log2 of its largest |Re|, |Im| over its RMS scalar,
// log2(r) + log2 sqrt(2 len) - log2 ||v|| with ||v||^2 = sh 2^(2e); 0 for a zero vector
__device__ __forceinline__ double crest_of(double r, int e, double sh, int len) {
  if (!(r > 0.0)) return 0.0;
  const double half_l2k = 0.5 * log2(2.0 * len);
  return log2(ldexp(r, -e)) + half_l2k - 0.5 * log2(sh);
}

// op(M) = M: vector i is row i, entries M[i + l ld] -- one thread per vector (coalesced)
__global__ void vec_stats_rows_kernel(const double2* M, long long ld, int count, int len, SelVecStats out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double r = 0.0;
  int z = 0;
  for (int l = 0; l < len; ++l) {
    const double2 v = M[i + l * ld];
    r = fmax(r, fmax(fabs(v.x), fabs(v.y)));
    z += (v.x == 0.0 && v.y == 0.0);
  }
  const int e = frexp_exp(r);
  double sh = 0.0;
  for (int l = 0; l < len; ++l) {
    const double2 v = M[i + l * ld];
    const double a = ldexp(v.x, -e), b = ldexp(v.y, -e);
    sh += a * a + b * b;
  }
  out.r[i] = r;
  out.e[i] = e;
  out.sh[i] = sh;
  out.z[i] = z;
  out.cr[i] = crest_of(r, e, sh, len);
}

// op(M) = M^T or M^H: vector i is column i of M, contiguous -- one warp per vector
__global__ void vec_stats_cols_kernel(const double2* M, long long ld, int count, int len, SelVecStats out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= count) return;
  const double2* col = M + w * ld;
  double r = 0.0;
  int z = 0;
  for (int l = lane; l < len; l += 32) {
    const double2 v = col[l];
    r = fmax(r, fmax(fabs(v.x), fabs(v.y)));
    z += (v.x == 0.0 && v.y == 0.0);
  }
  for (int o = 16; o; o >>= 1) {
    r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
  const int e = frexp_exp(r);
  double sh = 0.0;
  for (int l = lane; l < len; l += 32) {
    const double2 v = col[l];
    const double a = ldexp(v.x, -e), b = ldexp(v.y, -e);
    sh += a * a + b * b;
  }
  for (int o = 16; o; o >>= 1) sh += __shfl_xor_sync(0xffffffffu, sh, o);
  if (lane == 0) {
    out.r[w] = r;
    out.e[w] = e;
    out.sh[w] = sh;
    out.z[w] = z;
    out.cr[w] = crest_of(r, e, sh, len);
  }
}

// EA = max e over the nonzero rows of op(A), EB likewise over op(B)'s columns (0 if none).
__global__ void max_exp_kernel(SelVecStats a, int ma, SelVecStats b, int nb, int* ex) {
  __shared__ int sa[256], sb[256];
  int xa = INT_MIN, xb = INT_MIN;
  for (int i = threadIdx.x; i < ma; i += blockDim.x)
    if (a.r[i] > 0.0) xa = max(xa, a.e[i]);
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (b.r[i] > 0.0) xb = max(xb, b.e[i]);
  sa[threadIdx.x] = xa;
  sb[threadIdx.x] = xb;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] = max(sa[threadIdx.x], sa[threadIdx.x + s]);
      sb[threadIdx.x] = max(sb[threadIdx.x], sb[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ex[0] = sa[0] == INT_MIN ? 0 : sa[0];
    ex[1] = sb[0] == INT_MIN ? 0 : sb[0];
  }
}

// ------------------------------------------------------------------ compensated complex GEMV
// Y (rows x SEL_PROBES) = (2^-E op(M)) X with X = Xh + Xl given as a double-double (Xl may be
// null) and Y returned as a double-double Yh + Yl.  The sums use the compensated dot product
// of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005): every
// product is split exactly by an FMA, every addition by the error-free two-sum, and the
// errors are summed separately, so the result is as accurate as a computation in twice the
// working precision.  The intrinsics keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// (s, c) += a * b
__device__ __forceinline__ void dot2(double& s, double& c, double a, double b) {
  const double p = __dmul_rn(a, b);
  const double e = __fma_rn(a, b, -p);
  double q;
  two_sum(s, p, s, q);
  c = __dadd_rn(c, __dadd_rn(q, e));
}

// (s, c) += (sb, cb)
__device__ __forceinline__ void dd_add(double& s, double& c, double sb, double cb) {
  double q;
  two_sum(s, sb, s, q);
  c = __dadd_rn(c, __dadd_rn(q, cb));
}

// complex accumulators (re: s, c; im: s, c) for one probe
struct CAcc { double rs, rc, is, ic; };

// acc += a * (xh + xl) for complex a and double-double x
__device__ __forceinline__ void cmac(CAcc& A, double ar, double ai, double2 xh, double2 xl) {
  dot2(A.rs, A.rc, ar, xh.x);
  dot2(A.rs, A.rc, -ai, xh.y);
  dot2(A.is, A.ic, ar, xh.y);
  dot2(A.is, A.ic, ai, xh.x);
  A.rc = __fma_rn(ar, xl.x, A.rc);
  A.rc = __fma_rn(-ai, xl.y, A.rc);
  A.ic = __fma_rn(ar, xl.y, A.ic);
  A.ic = __fma_rn(ai, xl.x, A.ic);
}

// normalised double-double of an accumulator
__device__ __forceinline__ void cacc_out(const CAcc& A, double2& h, double2& l) {
  double e;
  two_sum(A.rs, A.rc, h.x, e);
  l.x = e;
  two_sum(A.is, A.ic, h.y, e);
  l.y = e;
}

constexpr int GEMV_CHUNK = 16;

// op(M) = M (rows strided): grid.x over blocks of 64 rows, grid.y over chunks of GEMV_CHUNK of
// the reduction, grid.z over the probes; each thread writes its row's partial double-double of
// its chunk and probe (short dependency chains across many blocks: the compensated sums run on
// the binary64 pipe).
// PLAIN: the chunk's products and sums in binary64 (fused multiply-adds, Xl ignored); the
// chunk partials are still added in double-double by gemv_reduce_kernel, so the result is off
// by at most about GEMV_CHUNK eps sum_l |m_l x_l| (the residual check's product W = D X, whose
// compensated sums ran on the binary64 pipe at four times the cost)
template <bool PLAIN>
__global__ void gemv_rows_kernel(const double2* M, long long ld, int rows, int len, const double2* Xh,
                                 const double2* Xl, int ldx, double2* part, const int* ex, int eidx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int E = ex ? ex[eidx] : 0;
  const int q = blockIdx.z;
  const int l0 = blockIdx.y * GEMV_CHUNK, l1 = min(len, l0 + GEMV_CHUNK);
  CAcc acc{0.0, 0.0, 0.0, 0.0};
  for (int l = l0; l < l1; ++l) {
    const double2 a = M[i + l * ld];
    const double ar = ldexp(a.x, -E), ai = ldexp(a.y, -E);
    if constexpr (PLAIN) {
      const double2 x = Xh[l + q * ldx];
      acc.rs = __fma_rn(ar, x.x, __fma_rn(-ai, x.y, acc.rs));
      acc.is = __fma_rn(ar, x.y, __fma_rn(ai, x.x, acc.is));
    } else {
      cmac(acc, ar, ai, Xh[l + q * ldx], Xl ? Xl[l + q * ldx] : make_double2(0.0, 0.0));
    }
  }
  // part[chunk][q][row] as (s re, s im) then (c re, c im)
  const long long o = 2 * ((static_cast<long long>(blockIdx.y) * SEL_PROBES + q) * rows + i);
  part[o] = make_double2(acc.rs, acc.is);
  part[o + 1] = make_double2(acc.rc, acc.ic);
}

// sum the chunks of gemv_rows_kernel in double-double: Y = Yh + Yl (rows x SEL_PROBES, ld
// rows); one warp per output, the lanes' partial sums combined by shuffles
__global__ void gemv_reduce_kernel(const double2* part, int rows, int nchunks, double2* Yh, double2* Yl) {
  const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= rows * SEL_PROBES) return;
  CAcc A{0.0, 0.0, 0.0, 0.0};
  for (int c = lane; c < nchunks; c += 32) {
    const long long o = 2 * (static_cast<long long>(c) * SEL_PROBES * rows + idx);
    const double2 sv = part[o], cv = part[o + 1];
    dd_add(A.rs, A.rc, sv.x, cv.x);
    dd_add(A.is, A.ic, sv.y, cv.y);
  }
  for (int o = 16; o; o >>= 1) {
    const double rs = __shfl_xor_sync(0xffffffffu, A.rs, o), rc = __shfl_xor_sync(0xffffffffu, A.rc, o);
    const double is = __shfl_xor_sync(0xffffffffu, A.is, o), ic = __shfl_xor_sync(0xffffffffu, A.ic, o);
    dd_add(A.rs, A.rc, rs, rc);
    dd_add(A.is, A.ic, is, ic);
  }
  if (lane == 0) cacc_out(A, Yh[idx], Yl[idx]);
}

// op(M) = M^T or M^H (row i of op(M) is column i of M, contiguous): one warp per row
__global__ void gemv_cols_kernel(const double2* M, long long ld, int rows, int len, int conj, const double2* Xh,
                                 const double2* Xl, int ldx, double2* Yh, double2* Yl, int ldy, const int* ex,
                                 int eidx) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const int E = ex ? ex[eidx] : 0;
  const double2* col = M + w * ld;
  CAcc acc[SEL_PROBES];
#pragma unroll
  for (int q = 0; q < SEL_PROBES; ++q) acc[q] = CAcc{0.0, 0.0, 0.0, 0.0};
  for (int l = lane; l < len; l += 32) {
    const double2 a = col[l];
    const double ar = ldexp(a.x, -E), ai = conj ? -ldexp(a.y, -E) : ldexp(a.y, -E);
#pragma unroll
    for (int q = 0; q < SEL_PROBES; ++q)
      cmac(acc[q], ar, ai, Xh[l + q * ldx], Xl ? Xl[l + q * ldx] : make_double2(0.0, 0.0));
  }
#pragma unroll
  for (int q = 0; q < SEL_PROBES; ++q)
    for (int o = 16; o; o >>= 1) {
      const double rs = __shfl_xor_sync(0xffffffffu, acc[q].rs, o), rc = __shfl_xor_sync(0xffffffffu, acc[q].rc, o);
      const double is = __shfl_xor_sync(0xffffffffu, acc[q].is, o), ic = __shfl_xor_sync(0xffffffffu, acc[q].ic, o);
      dd_add(acc[q].rs, acc[q].rc, rs, rc);
      dd_add(acc[q].is, acc[q].ic, is, ic);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < SEL_PROBES; ++q) cacc_out(acc[q], Yh[w + q * ldy], Yl[w + q * ldy]);
}

// ------------------------------------------------------------------ feature reduction
// One block of 256 threads, binary64 block reductions in a fixed order.
constexpr int RED_T = 256;

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RED_T / 2; s; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RED_T / 2; s; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

struct CrestStats { double mean, max, std, espread, log2sum_sh, log2sum_one, count; };

// Statistics of the nonzero vectors of one operand (see the feature list below).  Emax is the
// operand's max exponent (ex[]).
__device__ CrestStats crest_stats(const SelVecStats v, int count, int Emax, double* sh) {
  CrestStats c{0, 0, 0, 0, -INFINITY, -INFINITY, 0};
  double n = 0, s = 0, mx = -INFINITY, se = 0, ssh = 0, sone = 0;
  for (int i = threadIdx.x; i < count; i += RED_T) {
    const double r = v.r[i];
    if (r > 0.0) {
      const int e = v.e[i];
      const double cr = v.cr[i];
      n += 1;
      s += cr;
      mx = fmax(mx, cr);
      se += e;
      ssh += ldexp(v.sh[i], 2 * (e - Emax));
      sone += ldexp(1.0, 2 * (e - Emax));
    }
  }
  n = block_sum(n, sh);
  if (n == 0) return c;
  s = block_sum(s, sh);
  mx = block_max(mx, sh);
  se = block_sum(se, sh);
  ssh = block_sum(ssh, sh);
  sone = block_sum(sone, sh);
  const double mean = s / n;
  double d2 = 0;
  for (int i = threadIdx.x; i < count; i += RED_T) {
    if (v.r[i] > 0.0) {
      const double cr = v.cr[i];
      d2 += (cr - mean) * (cr - mean);
    }
  }
  d2 = block_sum(d2, sh);
  c.mean = mean;
  c.max = mx;
  c.std = sqrt(d2 / n);
  c.espread = static_cast<double>(Emax) - se / n;
  c.log2sum_sh = 2.0 * Emax + log2(ssh);
  c.log2sum_one = 2.0 * Emax + log2(sone);
  c.count = n;
  return c;
}

// Features of op(A) op(B) (m x k times k x n) from the vector statistics, the probes X and
// the scaled probe product zs = (2^-EA op(A)) ((2^-EB op(B)) X):
//   f0..f2  = log2 k, log2 m, log2 n (each / 10)
//   crest of a vector: log2(r 2^-e) + log2(2k)/2 - log2(sh)/2
//   f3..f5  = mean, max, population std of the crest over op(A)'s nonzero rows (/ 8)
//   f6..f8  = the same over op(B)'s nonzero columns (/ 8)
//   f9, f10 = (max e - mean e) / 16 over those rows / columns
//   log2 c  = log2(n ||zs||^2 / ||X||^2) / 2 + EA + EB
//   lA = log2 sum sh_i 4^e_i = log2 ||op(A)||_F^2, lB likewise
//   f11 = (lA/2 + lB/2 - log2 c) / 16
//   f12 = (log2(2^(log2 sum 4^e_i + lB) + 2^(log2 sum 4^f_j + lA)) / 2 - log2 c) / 16
//   f13, f14 = fractions of exactly zero entries; f15 = 1
// f11, f12 = 0 when zs = 0 or an operand is zero.  Also stores E = EA + EB and ||zs||^2.
__global__ void __launch_bounds__(RED_T) selector_features_kernel(SelVecStats a, int m, SelVecStats b, int n, int k,
                                                                  const double2* X, const double2* zs, const int* ex,
                                                                  float* f, SelAux* aux) {
  // zs: the leading parts of the double-double probe product
  __shared__ double sh[RED_T];
  const int EA = ex[0], EB = ex[1];
  const CrestStats ca = crest_stats(a, m, EA, sh);
  const CrestStats cb = crest_stats(b, n, EB, sh);
  double z2 = 0, x2 = 0, za = 0, zb = 0;
  for (int i = threadIdx.x; i < m * SEL_PROBES; i += RED_T) z2 += zs[i].x * zs[i].x + zs[i].y * zs[i].y;
  for (int i = threadIdx.x; i < n * SEL_PROBES; i += RED_T) x2 += X[i].x * X[i].x + X[i].y * X[i].y;
  for (int i = threadIdx.x; i < m; i += RED_T) za += a.z[i];
  for (int i = threadIdx.x; i < n; i += RED_T) zb += b.z[i];
  z2 = block_sum(z2, sh);
  x2 = block_sum(x2, sh);
  za = block_sum(za, sh);
  zb = block_sum(zb, sh);
  if (threadIdx.x == 0) {
    double F[SEL_NF];
    F[0] = log2(static_cast<double>(max(k, 1))) / 10;
    F[1] = log2(static_cast<double>(max(m, 1))) / 10;
    F[2] = log2(static_cast<double>(max(n, 1))) / 10;
    F[3] = ca.mean / 8; F[4] = ca.count > 0 ? ca.max / 8 : 0.0; F[5] = ca.std / 8;
    F[6] = cb.mean / 8; F[7] = cb.count > 0 ? cb.max / 8 : 0.0; F[8] = cb.std / 8;
    F[9] = ca.espread / 16;
    F[10] = cb.espread / 16;
    F[11] = 0.0;
    F[12] = 0.0;
    if (z2 > 0.0 && ca.count > 0 && cb.count > 0) {
      const double lc = 0.5 * log2(n * z2 / x2) + EA + EB;
      const double lA = ca.log2sum_sh, lB = cb.log2sum_sh;
      F[11] = (0.5 * lA + 0.5 * lB - lc) / 16;
      const double ta = ca.log2sum_one + lB, tb = cb.log2sum_one + lA;
      const double hi = fmax(ta, tb);
      F[12] = (0.5 * (hi + log2(exp2(ta - hi) + exp2(tb - hi))) - lc) / 16;
    }
    F[13] = za / fmax(1.0, static_cast<double>(m) * k);
    F[14] = zb / fmax(1.0, static_cast<double>(k) * n);
    F[15] = 1.0;
    for (int i = 0; i < SEL_NF; ++i) f[i] = static_cast<float>(F[i]);
    aux->E = EA + EB;
    aux->z2 = z2;
  }
}

// residual: r^2 = ||2^-E W - zs||^2 / ||zs||^2 with W = D X (m x SEL_PROBES), both
// double-doubles, the difference formed before it is rounded
// (block partials of num and den into rpart, then residual_final_kernel sums them in order)
__global__ void __launch_bounds__(RED_T) residual_kernel(const double2* Wh, const double2* Wl, const double2* zh,
                                                         const double2* zl, int m, SelAux* aux, double* rpart) {
  __shared__ double sh[RED_T];
  const int E = aux->E;
  double num = 0, den = 0;
  for (int i = blockIdx.x * RED_T + threadIdx.x; i < m * SEL_PROBES; i += gridDim.x * RED_T) {
    double dx, ex, dy, ey;
    two_sum(ldexp(Wh[i].x, -E), -zh[i].x, dx, ex);
    two_sum(ldexp(Wh[i].y, -E), -zh[i].y, dy, ey);
    dx = dx + (ex + (ldexp(Wl[i].x, -E) - zl[i].x));
    dy = dy + (ey + (ldexp(Wl[i].y, -E) - zl[i].y));
    num += dx * dx + dy * dy;
    den += zh[i].x * zh[i].x + zh[i].y * zh[i].y;
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) {
    rpart[2 * blockIdx.x] = num;
    rpart[2 * blockIdx.x + 1] = den;
  }
}

__global__ void __launch_bounds__(RED_T) residual_final_kernel(const double* rpart, int nblocks, SelAux* aux) {
  __shared__ double sh[RED_T];
  double num = 0, den = 0;
  for (int b = threadIdx.x; b < nblocks; b += RED_T) {
    num += rpart[2 * b];
    den += rpart[2 * b + 1];
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) aux->resid = den > 0.0 ? sqrt(num / den) : (num == 0.0 ? 0.0 : INFINITY);
}

// relative Frobenius difference ||X - Y|| / ||Y|| of two m x n matrices: per-column partial
// sums, then one block
__global__ void diff_cols_kernel(int m, int n, const double2* X, long long ldx, const double2* Y, long long ldy,
                                 double* part) {
  const int j = blockIdx.x;
  __shared__ double sh[RED_T];
  double num = 0, den = 0;
  for (int i = threadIdx.x; i < m; i += RED_T) {
    const double2 x = X[i + j * ldx], y = Y[i + j * ldy];
    const double dx = x.x - y.x, dy = x.y - y.y;
    num += dx * dx + dy * dy;
    den += y.x * y.x + y.y * y.y;
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) {
    part[2 * j] = num;
    part[2 * j + 1] = den;
  }
}

__global__ void diff_final_kernel(int n, const double* part, double* out) {
  __shared__ double sh[RED_T];
  double num = 0, den = 0;
  for (int j = threadIdx.x; j < n; j += RED_T) {
    num += part[2 * j];
    den += part[2 * j + 1];
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) out[0] = den > 0.0 ? sqrt(num / den) : (num == 0.0 ? 0.0 : INFINITY);
}

// C = alpha D + beta C (complex binary64, column major)
__global__ void axpby_kernel(int m, int n, const double2* D, long long ldd, double2* C, long long ldc, double ar,
                             double ai, double br, double bi) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(m) * n) return;
  const int i = static_cast<int>(idx % m), j = static_cast<int>(idx / m);
  const double2 d = D[i + j * ldd];
  double2 c = C[i + j * ldc];
  double2 o;
  if (br == 0.0 && bi == 0.0) c = make_double2(0.0, 0.0);
  o.x = ar * d.x - ai * d.y + br * c.x - bi * c.y;
  o.y = ar * d.y + ai * d.x + br * c.y + bi * c.x;
  C[i + j * ldc] = o;
}

// ------------------------------------------------------------------ the perceptron (float32)
constexpr int OFF_W1 = 0, OFF_B1 = SEL_NH * SEL_NF, OFF_W2 = OFF_B1 + SEL_NH, OFF_B2 = OFF_W2 + SEL_NH * SEL_NH,
              OFF_W3 = OFF_B2 + SEL_NH, OFF_B3 = OFF_W3 + SEL_NO * SEL_NH;
static_assert(OFF_B3 + SEL_NO == SEL_NPARAMS, "parameter layout");

__device__ __forceinline__ void load_params(const float* P, float* w) {
  for (int i = threadIdx.x; i < SEL_NPARAMS; i += blockDim.x) w[i] = P[i];
  __syncthreads();
}

// Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per sample (row of X, N x 16); stores the
// pre-activations Z1, Z2 (N x 64 each) when asked.
__global__ void mlp_forward_kernel(const float* P, const float* X, int N, float* Z1, float* Z2, float* Y) {
  __shared__ float w[SEL_NPARAMS];
  load_params(P, w);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  float x[SEL_NF], h1[SEL_NH], y[SEL_NO];
#pragma unroll
  for (int i = 0; i < SEL_NF; ++i) x[i] = X[s * SEL_NF + i];
#pragma unroll
  for (int j = 0; j < SEL_NH; ++j) {
    float z = w[OFF_B1 + j];
#pragma unroll
    for (int i = 0; i < SEL_NF; ++i) z = fmaf(w[OFF_W1 + j * SEL_NF + i], x[i], z);
    if (Z1) Z1[s * SEL_NH + j] = z;
    h1[j] = fmaxf(z, 0.0f);
  }
#pragma unroll
  for (int o = 0; o < SEL_NO; ++o) y[o] = w[OFF_B3 + o];
  for (int j = 0; j < SEL_NH; ++j) {
    float z = w[OFF_B2 + j];
#pragma unroll
    for (int i = 0; i < SEL_NH; ++i) z = fmaf(w[OFF_W2 + j * SEL_NH + i], h1[i], z);
    if (Z2) Z2[s * SEL_NH + j] = z;
    const float h = fmaxf(z, 0.0f);
#pragma unroll
    for (int o = 0; o < SEL_NO; ++o) y[o] = fmaf(w[OFF_W3 + o * SEL_NH + j], h, y[o]);
  }
#pragma unroll
  for (int o = 0; o < SEL_NO; ++o) Y[s * SEL_NO + o] = y[o];
}

// dY = 2 (Y - T) / (8 N); dZ2 = (W3^T dY) * [Z2 > 0]; dZ1 = (W2^T dZ2) * [Z1 > 0]
__global__ void mlp_backward_kernel(const float* P, const float* Z1, const float* Z2, const float* Y, const float* T,
                                    int N, float* dY, float* dZ2, float* dZ1) {
  __shared__ float w[SEL_NPARAMS];
  load_params(P, w);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const float scale = 2.0f / (static_cast<float>(N) * SEL_NO);
  float dy[SEL_NO], dh1[SEL_NH];
#pragma unroll
  for (int o = 0; o < SEL_NO; ++o) {
    dy[o] = scale * (Y[s * SEL_NO + o] - T[s * SEL_NO + o]);
    dY[s * SEL_NO + o] = dy[o];
  }
#pragma unroll
  for (int i = 0; i < SEL_NH; ++i) dh1[i] = 0.0f;
  for (int j = 0; j < SEL_NH; ++j) {
    float d = 0.0f;
#pragma unroll
    for (int o = 0; o < SEL_NO; ++o) d = fmaf(w[OFF_W3 + o * SEL_NH + j], dy[o], d);
    d = Z2[s * SEL_NH + j] > 0.0f ? d : 0.0f;
    dZ2[s * SEL_NH + j] = d;
#pragma unroll
    for (int i = 0; i < SEL_NH; ++i) dh1[i] = fmaf(w[OFF_W2 + j * SEL_NH + i], d, dh1[i]);
  }
#pragma unroll
  for (int i = 0; i < SEL_NH; ++i) dZ1[s * SEL_NH + i] = Z1[s * SEL_NH + i] > 0.0f ? dh1[i] : 0.0f;
}

// One thread per parameter: the gradient summed over the samples in order.
__global__ void mlp_grad_kernel(const float* X, const float* Z1, const float* Z2, const float* dY, const float* dZ2,
                                const float* dZ1, int N, float* g) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= SEL_NPARAMS) return;
  float acc = 0.0f;
  if (q < OFF_B1) {
    const int j = q / SEL_NF, i = q % SEL_NF;
    for (int s = 0; s < N; ++s) acc = fmaf(dZ1[s * SEL_NH + j], X[s * SEL_NF + i], acc);
  } else if (q < OFF_W2) {
    const int j = q - OFF_B1;
    for (int s = 0; s < N; ++s) acc += dZ1[s * SEL_NH + j];
  } else if (q < OFF_B2) {
    const int j = (q - OFF_W2) / SEL_NH, i = (q - OFF_W2) % SEL_NH;
    for (int s = 0; s < N; ++s) acc = fmaf(dZ2[s * SEL_NH + j], fmaxf(Z1[s * SEL_NH + i], 0.0f), acc);
  } else if (q < OFF_W3) {
    const int j = q - OFF_B2;
    for (int s = 0; s < N; ++s) acc += dZ2[s * SEL_NH + j];
  } else if (q < OFF_B3) {
    const int o = (q - OFF_W3) / SEL_NH, j = (q - OFF_W3) % SEL_NH;
    for (int s = 0; s < N; ++s) acc = fmaf(dY[s * SEL_NO + o], fmaxf(Z2[s * SEL_NH + j], 0.0f), acc);
  } else {
    const int o = q - OFF_B3;
    for (int s = 0; s < N; ++s) acc += dY[s * SEL_NO + o];
  }
  g[q] = acc;
}

// Adam with bias correction; t = step number (>= 1).
__global__ void adam_kernel(float* P, const float* g, float* m, float* v, int t, float lr, float b1, float b2,
                            float eps) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= SEL_NPARAMS) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.0f - b1) * gq;
  const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float mh = mq / (1.0f - powf(b1, static_cast<float>(t)));
  const float vh = vq / (1.0f - powf(b2, static_cast<float>(t)));
  P[q] -= lr * mh / (sqrtf(vh) + eps);
}

// mean squared error over N x 8 outputs (binary64 accumulation in a fixed order)
__global__ void __launch_bounds__(RED_T) mse_kernel(const float* Y, const float* T, int N, double* out) {
  __shared__ double sh[RED_T];
  double s = 0;
  for (int i = threadIdx.x; i < N * SEL_NO; i += RED_T) {
    const double d = static_cast<double>(Y[i]) - static_cast<double>(T[i]);
    s += d * d;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s / (static_cast<double>(N) * SEL_NO);
}

// smallest S in 3..10 with prediction <= lim, else 10; aux->S and the predictions
__global__ void choose_kernel(const float* Y, float lim, SelAux* aux) {
  if (threadIdx.x) return;
  int S = SEL_SMAX;
  for (int o = 0; o < SEL_NO; ++o) {
    aux->pred[o] = Y[o];
    if (S == SEL_SMAX && Y[o] <= lim) S = SEL_SMIN + o;
  }
  aux->S = S;
}

// deferred check of one GEMM of a solve (S its slice count): no host read in between
__global__ void defer_check_kernel(const SelAux* aux, int S, int with_pred, double pass, SelDefer* rec) {
  if (threadIdx.x) return;
  const double r = aux->resid;
  if (!(r <= pass)) rec->failed = 1;
  if (S >= SEL_SMIN && S <= SEL_SMAX) rec->count[S - SEL_SMIN] += 1;
  if (!(r <= rec->max_resid)) rec->max_resid = r;
  if (with_pred)
    for (int o = 0; o < SEL_NO; ++o) rec->pred[o] = aux->pred[o];
}

// ------------------------------------------------------------------ launchers
static unsigned blocks(long long n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

void launch_probe(double2* X, int n, const SelBases& b, cudaStream_t st) {
  probe_kernel<<<blocks(n, 256), 256, 0, st>>>(X, n, b);
  record_launch();
}

void launch_vec_stats(const double2* M, long long ld, int count, int len, bool contiguous, const SelVecStats& out,
                      cudaStream_t st) {
  if (count <= 0) return;
  if (contiguous)
    vec_stats_cols_kernel<<<blocks(static_cast<long long>(count) * 32, 256), 256, 0, st>>>(M, ld, count, len, out);
  else
    vec_stats_rows_kernel<<<blocks(count, 128), 128, 0, st>>>(M, ld, count, len, out);
  record_launch();
}

void launch_max_exp(const SelVecStats& a, int ma, const SelVecStats& b, int nb, int* ex, cudaStream_t st) {
  max_exp_kernel<<<1, 256, 0, st>>>(a, ma, b, nb, ex);
  record_launch();
}

int gemv_chunks(int len) { return (len + GEMV_CHUNK - 1) / GEMV_CHUNK; }

void launch_gemv(const double2* M, long long ld, int rows, int len, int op, const double2* Xh, const double2* Xl,
                 int ldx, double2* Yh, double2* Yl, double2* part, const int* ex, int eidx, cudaStream_t st,
                 bool plain) {
  if (rows <= 0) return;
  if (op == 0) {
    const int nch = std::max(1, gemv_chunks(len));
    const dim3 grid(blocks(rows, 64), nch, SEL_PROBES);
    if (plain) gemv_rows_kernel<true><<<grid, 64, 0, st>>>(M, ld, rows, len, Xh, Xl, ldx, part, ex, eidx);
    else gemv_rows_kernel<false><<<grid, 64, 0, st>>>(M, ld, rows, len, Xh, Xl, ldx, part, ex, eidx);
    record_launch();
    gemv_reduce_kernel<<<blocks(static_cast<long long>(rows) * SEL_PROBES * 32, 256), 256, 0, st>>>(part, rows, nch,
                                                                                                   Yh, Yl);
  } else {
    gemv_cols_kernel<<<blocks(static_cast<long long>(rows) * 32, 256), 256, 0, st>>>(M, ld, rows, len, op == 2, Xh,
                                                                                     Xl, ldx, Yh, Yl, rows, ex, eidx);
  }
  record_launch();
}

void launch_selector_features(const SelVecStats& a, int m, const SelVecStats& b, int n, int k, const double2* X,
                              const double2* zs, const int* ex, float* f, SelAux* aux, cudaStream_t st) {
  selector_features_kernel<<<1, RED_T, 0, st>>>(a, m, b, n, k, X, zs, ex, f, aux);
  record_launch();
}

void launch_residual(const double2* Wh, const double2* Wl, const double2* zh, const double2* zl, int m, SelAux* aux,
                     double* rpart, cudaStream_t st) {
  const int nb = static_cast<int>(std::min<long long>(256, blocks(static_cast<long long>(m) * SEL_PROBES, RED_T)));
  residual_kernel<<<nb, RED_T, 0, st>>>(Wh, Wl, zh, zl, m, aux, rpart);
  record_launch();
  residual_final_kernel<<<1, RED_T, 0, st>>>(rpart, nb, aux);
  record_launch();
}

void launch_rel_diff(int m, int n, const double2* X, long long ldx, const double2* Y, long long ldy, double* part,
                     double* out, cudaStream_t st) {
  diff_cols_kernel<<<n, RED_T, 0, st>>>(m, n, X, ldx, Y, ldy, part);
  record_launch();
  diff_final_kernel<<<1, RED_T, 0, st>>>(n, part, out);
  record_launch();
}

void launch_axpby(int m, int n, const double2* D, long long ldd, double2* C, long long ldc, double ar, double ai,
                  double br, double bi, cudaStream_t st) {
  const long long tot = static_cast<long long>(m) * n;
  if (tot == 0) return;
  axpby_kernel<<<blocks(tot, 256), 256, 0, st>>>(m, n, D, ldd, C, ldc, ar, ai, br, bi);
  record_launch();
}

void launch_mlp_forward(const float* P, const float* X, int N, float* Z1, float* Z2, float* Y, cudaStream_t st) {
  if (N <= 0) return;
  mlp_forward_kernel<<<blocks(N, 128), 128, 0, st>>>(P, X, N, Z1, Z2, Y);
  record_launch();
}

void launch_mlp_train(float* P, float* gbuf, float* m, float* v, int t, float lr, const float* X, const float* T,
                      int N, float* Z1, float* Z2, float* Y, float* dY, float* dZ2, float* dZ1, double* loss,
                      cudaStream_t st) {
  mlp_forward_kernel<<<blocks(N, 128), 128, 0, st>>>(P, X, N, Z1, Z2, Y);
  record_launch();
  mse_kernel<<<1, RED_T, 0, st>>>(Y, T, N, loss);
  record_launch();
  mlp_backward_kernel<<<blocks(N, 128), 128, 0, st>>>(P, Z1, Z2, Y, T, N, dY, dZ2, dZ1);
  record_launch();
  mlp_grad_kernel<<<blocks(SEL_NPARAMS, 128), 128, 0, st>>>(X, Z1, Z2, dY, dZ2, dZ1, N, gbuf);
  record_launch();
  adam_kernel<<<blocks(SEL_NPARAMS, 256), 256, 0, st>>>(P, gbuf, m, v, t, lr, 0.9f, 0.999f, 1e-8f);
  record_launch();
}

void launch_mlp_grad_only(const float* P, float* gbuf, const float* X, const float* T, int N, float* Z1, float* Z2,
                          float* Y, float* dY, float* dZ2, float* dZ1, cudaStream_t st) {
  mlp_forward_kernel<<<blocks(N, 128), 128, 0, st>>>(P, X, N, Z1, Z2, Y);
  record_launch();
  mlp_backward_kernel<<<blocks(N, 128), 128, 0, st>>>(P, Z1, Z2, Y, T, N, dY, dZ2, dZ1);
  record_launch();
  mlp_grad_kernel<<<blocks(SEL_NPARAMS, 128), 128, 0, st>>>(X, Z1, Z2, dY, dZ2, dZ1, N, gbuf);
  record_launch();
}

// log10 of a relative error, floored at 1e-17 (training targets of the selector)
__global__ void log_err_kernel(const double* rel, float* dst) {
  const double r = *rel;
  dst[0] = r > 1e-17 ? static_cast<float>(log10(r)) : -17.0f;
}

void launch_log_err(const double* rel, float* dst, cudaStream_t st) {
  log_err_kernel<<<1, 1, 0, st>>>(rel, dst);
  record_launch();
}

void launch_choose(const float* Y, float lim, SelAux* aux, cudaStream_t st) {
  choose_kernel<<<1, 32, 0, st>>>(Y, lim, aux);
  record_launch();
}

void launch_defer_check(const SelAux* aux, int S, bool with_pred, double pass, SelDefer* rec, cudaStream_t st) {
  defer_check_kernel<<<1, 32, 0, st>>>(aux, S, with_pred ? 1 : 0, pass, rec);
  record_launch();
}

}  // namespace ozk
