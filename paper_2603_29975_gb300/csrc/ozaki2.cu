// Ozaki-II (CRT) emulation kernels (paper Sec. 2.2: convert the matrices to integers, multiply
// them modulo several small pairwise-coprime moduli, reconstruct with the Chinese Remainder
// Theorem; the precision knob is the number of moduli, Sec. 3.2 and Sec. 4).
//   * residue_split_kernel: per row of op(A) (column of op(B)) the frexp exponent of the max
//     over |Re|, |Im|, the integer image X = trunc(x 2^(beta - e)) (|X| < 2^beta, beta <= 63),
//     and for every modulus m the symmetric residue of X in (-m/2, m/2], written as fp16 in the
//     stacked layout of the slice split (one plane per modulus).  The residue is formed from the
//     balanced base-256 digits of X: X mod m = sum_s d_s (256^s mod m) mod m, small integers only.
//   * the products of the residue planes run in slice_gemm_kernel (one pair per modulus, its
//     exact integer value added to an int32 buffer per modulus);
//   * crt_kernel: per output the residues of the N exact products, Garner's mixed-radix digits
//     v_t = (r_t - sum_{j<t} v_j (m_0...m_{j-1} mod m_t)) (m_0...m_{t-1})^-1 mod m_t, the value
//     sum_t v_t m_0...m_{t-1} in [0, P) by Horner in 128-bit integers, the symmetric lift to
//     (-P/2, P/2], the scaling 2^(e_i + f_j - 2 beta) with one rounding to binary64, and the
//     alpha / beta combination.
#include "ozk_params.cuh"

namespace ozk {

constexpr int RS_ROWS = 32;
constexpr int RS_THREADS = 256;

__device__ __forceinline__ int sym_mod(int v, int m) {
  int r = v % m;
  if (r < 0) r += m;
  return 2 * r > m ? r - m : r;
}

__global__ void __launch_bounds__(RS_THREADS) residue_split_kernel(const SplitParams p, const Oz2Tables T) {
  const int z = blockIdx.y;
  const bool single = p.X == nullptr;
  const int R = single ? p.rows1 : p.rows[z];
  const int K = single ? p.k1 : p.kdim[z];
  const int r0 = blockIdx.x * RS_ROWS;
  if (r0 >= R) return;
  const double2* __restrict__ P = single ? p.X1 + z * p.zstride1 : p.X[z];
  const long long ld = single ? p.ld1 : p.ld[z];
  const int tid = threadIdx.x;
  __shared__ unsigned long long rowmax[RS_ROWS];
  __shared__ int rowexp[RS_ROWS];
  __shared__ int bad;
  if (tid < RS_ROWS) rowmax[tid] = 0ull;
  if (tid == 0) bad = 0;
  __syncthreads();
  {
    int rl, l0, lstep;
    if (!p.trans) { rl = tid % RS_ROWS; l0 = tid / RS_ROWS; lstep = RS_THREADS / RS_ROWS; }
    else          { rl = tid / 8;       l0 = tid % 8;       lstep = 8; }
    const int r = r0 + rl;
    unsigned long long mx = 0ull;
    if (r < R) {
      for (int l = l0; l < K; l += lstep) {
        const double2 v = p.trans ? P[l + r * ld] : P[r + l * ld];
        const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v.x)) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v.y)) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long m2 = a > b ? a : b;
        if (m2 >= 0x7FF0000000000000ull) bad = 1;
        mx = m2 > mx ? m2 : mx;
      }
      atomicMax(&rowmax[rl], mx);
    }
  }
  __syncthreads();
  if (bad && tid == 0) flag_error(p.status, OZK_ERR_NONFINITE);
  if (tid < RS_ROWS) {
    const unsigned long long a = rowmax[tid];
    const int e = (a >= 0x7FF0000000000000ull) ? 0 : frexp_exponent_from_bits(a);
    rowexp[tid] = e;
    if (r0 + tid < R) p.exps[z * p.exp_stride + r0 + tid] = e;
  }
  __syncthreads();
  const int N = T.N;
  const long long plane = p.out_rows * p.kpad;
  __half* outz = p.out + static_cast<long long>(z) * N * plane;
  const int nr = min(RS_ROWS, R - r0);
  // stored row-fastest (trans == 0: rows of 32 consecutive threads) or column-fastest
  const int span = p.trans ? nr * K : RS_ROWS * K;
  for (int idx = tid; idx < span; idx += RS_THREADS) {
    int rl, l;
    if (!p.trans) { rl = idx % RS_ROWS; l = idx / RS_ROWS; if (rl >= nr) continue; }
    else          { rl = idx / K;       l = idx % K; }
    const int r = r0 + rl;
    // bit operations only (no binary64 compares or negations on the FP64 pipe); a non-finite
    // scalar (already flagged) is split as zero
    longlong2 v = reinterpret_cast<const longlong2*>(P)[p.trans ? l + r * ld : r + l * ld];
    if (p.conj) v.y ^= static_cast<long long>(0x8000000000000000ull);
    if ((v.x & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) v.x = 0;
    if ((v.y & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) v.y = 0;
    const int e = rowexp[rl];
    __int128 Xr = integer_image(__longlong_as_double(v.x), e, p.nbits);
    __int128 Xi = integer_image(__longlong_as_double(v.y), e, p.nbits);
    int dr[8], di[8];                                   // balanced base-256 digits, d[s] weight 256^s
#pragma unroll
    for (int s = 0; s < 7; ++s) { dr[s] = next_digit(Xr); di[s] = next_digit(Xi); }
    dr[7] = static_cast<int>(Xr);
    di[7] = static_cast<int>(Xi);
    for (int t = 0; t < N; ++t) {
      int ar = 0, ai = 0;
#pragma unroll
      for (int s = 0; s < 8; ++s) { ar += dr[s] * T.pow256[t][s]; ai += di[s] * T.pow256[t][s]; }
      const int rr = sym_mod(ar, T.mod[t]), ri = sym_mod(ai, T.mod[t]);
      __half* o = outz + t * plane;
      if (p.side == 0) {
        o[r * p.kpad + l] = __int2half_rn(rr);
        o[r * p.kpad + K + l] = __int2half_rn(ri);
      } else {
        const long long row0 = 2LL * r, row1 = 2LL * r + 1;
        o[row0 * p.kpad + l] = __int2half_rn(rr);
        o[row0 * p.kpad + K + l] = __int2half_rn(-ri);
        o[row1 * p.kpad + l] = __int2half_rn(ri);
        o[row1 * p.kpad + K + l] = __int2half_rn(rr);
      }
    }
  }
  // zero the K padding [2K, kpad) of the rows this CTA owns
  const int pad = static_cast<int>(p.kpad) - 2 * K;
  if (pad > 0) {
    const int rows_out = p.side == 0 ? 1 : 2;
    const int nro = nr * rows_out;
    for (int idx = tid; idx < N * nro * pad; idx += RS_THREADS) {
      const int c = idx % pad;
      const int rr = (idx / pad) % nro;
      const int t = idx / (pad * nro);
      outz[t * plane + (static_cast<long long>(r0) * rows_out + rr) * p.kpad + 2 * K + c] = __float2half(0.0f);
    }
  }
}

void launch_residue_split(const SplitParams& p, const Oz2Tables& T, int max_rows, int batch, cudaStream_t st) {
  dim3 grid((max_rows + RS_ROWS - 1) / RS_ROWS, batch);
  residue_split_kernel<<<grid, RS_THREADS, 0, st>>>(p, T);
  record_launch();
}

// value of the exact integer product congruent to res[t] mod m_t, in (-P/2, P/2]
__device__ __forceinline__ __int128 crt_value(const int* res, const Oz2Tables& T) {
  const int N = T.N;
  int v[OZ2_MAXMOD];
  for (int t = 0; t < N; ++t) {
    const int m = T.mod[t];
    int acc = res[t] % m;                               // |res| < 2^31: exact in int
    for (int j = 0; j < t; ++j) acc -= v[j] * T.pm[t][j] % m;
    acc %= m;
    if (acc < 0) acc += m;
    v[t] = static_cast<int>(static_cast<long long>(acc) * T.inv[t] % m);
  }
  // Horner: X = v_0 + m_0 (v_1 + m_1 (v_2 + ... ))
  unsigned __int128 X = static_cast<unsigned __int128>(v[N - 1]);
  for (int t = N - 2; t >= 0; --t) X = X * static_cast<unsigned>(T.mod[t]) + static_cast<unsigned>(v[t]);
  const unsigned __int128 P = (static_cast<unsigned __int128>(T.P_hi) << 64) | T.P_lo;
  return 2 * X > P ? -static_cast<__int128>(P - X) : static_cast<__int128>(X);
}

__global__ void crt_kernel(const CrtParams p, const Oz2Tables T) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long per = static_cast<long long>(p.m) * p.n;
  if (idx >= per * p.batch) return;
  const int z = static_cast<int>(idx / per);
  const long long rem = idx - z * per;
  const int i = static_cast<int>(rem % p.m), j = static_cast<int>(rem / p.m);
  int rre[OZ2_MAXMOD], rim[OZ2_MAXMOD];
  const int* base = p.R + static_cast<long long>(z) * T.N * p.plane + static_cast<long long>(i) * p.ldr;
  for (int t = 0; t < T.N; ++t) {
    rre[t] = base[t * p.plane + 2 * j];
    rim[t] = base[t * p.plane + 2 * j + 1];
  }
  const int E = p.e[z * p.e_stride + i] + p.f[z * p.f_stride + j] - 2 * p.beta;
  const double zr = round_scaled_dev(crt_value(rre, T), E);
  const double zi = round_scaled_dev(crt_value(rim, T), E);
  double2* dst = p.C + z * p.cstride + i + static_cast<long long>(j) * p.ldc;
  if (p.mode == EPI_STORE) {
    if (p.ar == 1.0 && p.ai == 0.0) *dst = make_double2(zr, zi);
    else *dst = make_double2(p.ar * zr - p.ai * zi, p.ar * zi + p.ai * zr);
  } else if (p.mode == EPI_LU) {
    const double2 c = *dst;
    *dst = make_double2(c.x - zr, c.y - zi);
  } else {
    const double2 c = *dst;
    const double xr = p.ar * zr - p.ai * zi, xi = p.ar * zi + p.ai * zr;
    *dst = make_double2(xr + p.br * c.x - p.bi * c.y, xi + p.br * c.y + p.bi * c.x);
  }
}

void launch_crt(const CrtParams& p, const Oz2Tables& T, cudaStream_t st) {
  const long long tot = static_cast<long long>(p.m) * p.n * p.batch;
  if (tot == 0) return;
  crt_kernel<<<static_cast<unsigned>((tot + 127) / 128), 128, 0, st>>>(p, T);
  record_launch();
}

}  // namespace ozk
