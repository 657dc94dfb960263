// Exponent scan and slice split (paper Sec. 2.2: slices by significant bits with exponent
// alignment).  One CTA owns 32 logical rows of an operand: it reads them once to find the
// per-row maximum of |Re| and |Im| (integer compare on the binary64 bit patterns), derives
// the frexp exponent, then reads them again (from L2) and writes the S balanced int8 digits
// of every real scalar as fp16 values in the K-major stacked layout the tensor-core kernel
// loads with TMA:
//   left operand  (side 0): out[z][s][r][l]     = digit of Re x_rl, out[z][s][r][k+l] = Im
//   right operand (side 1): out[z][s][2r][l]    = Re,  out[z][s][2r][k+l]   = -Im (digit-wise)
//                           out[z][s][2r+1][l]  = Im,  out[z][s][2r+1][k+l] = Re
// Positions [2k, kpad) of every written row are zero.  All integer work, no FP64 arithmetic.
#include <algorithm>
#include <type_traits>

#include "ozk_params.cuh"

namespace ozk {



constexpr int SPLIT_ROWS = 32;
constexpr int SPLIT_TK = 64;
constexpr int SPLIT_THREADS = 256;

// PER consecutive fp16 values (digits d[0..PER-1], negated when NEG) stored as one aligned
// vector at dst.
template <int PER, bool NEG>
__device__ __forceinline__ void store_digits(__half* dst, const int (&d)[PER]) {
  __half h[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) h[q] = __int2half_rn(NEG ? -d[q] : d[q]);
  if constexpr (PER == 8) {
    uint4 v;
    v.x = __half_as_ushort(h[0]) | (static_cast<uint32_t>(__half_as_ushort(h[1])) << 16);
    v.y = __half_as_ushort(h[2]) | (static_cast<uint32_t>(__half_as_ushort(h[3])) << 16);
    v.z = __half_as_ushort(h[4]) | (static_cast<uint32_t>(__half_as_ushort(h[5])) << 16);
    v.w = __half_as_ushort(h[6]) | (static_cast<uint32_t>(__half_as_ushort(h[7])) << 16);
    *reinterpret_cast<uint4*>(dst) = v;
  } else if constexpr (PER == 4) {
    uint2 v;
    v.x = __half_as_ushort(h[0]) | (static_cast<uint32_t>(__half_as_ushort(h[1])) << 16);
    v.y = __half_as_ushort(h[2]) | (static_cast<uint32_t>(__half_as_ushort(h[3])) << 16);
    *reinterpret_cast<uint2*>(dst) = v;
  } else if constexpr (PER == 2) {
    *reinterpret_cast<uint32_t*>(dst) = __half_as_ushort(h[0]) | (static_cast<uint32_t>(__half_as_ushort(h[1])) << 16);
  } else {
    *dst = h[0];
  }
}

// Digits of PER consecutive elements of one row (positions l .. l + PER - 1, all < K, l and K
// multiples of PER), every slice written with vector stores.  W64: 64-bit integer images
// (nbits <= 62), else 128-bit.
template <int PER, bool W64>
__device__ __forceinline__ void split_run(const SplitParams& p, const double2* v, int e, int r, int l, int K,
                                          __half* outz, long long plane) {
  using Int = typename std::conditional<W64, long long, __int128>::type;
  Int Xr[PER], Xi[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if constexpr (W64) {
      Xr[q] = integer_image64(v[q].x, e, p.nbits);
      Xi[q] = integer_image64(v[q].y, e, p.nbits);
    } else {
      Xr[q] = integer_image(v[q].x, e, p.nbits);
      Xi[q] = integer_image(v[q].y, e, p.nbits);
    }
  }
  for (int s = p.S - 1; s >= 0; --s) {
    int dr[PER], di[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      if constexpr (W64) {
        dr[q] = s ? next_digit64(Xr[q]) : static_cast<int>(Xr[q]);
        di[q] = s ? next_digit64(Xi[q]) : static_cast<int>(Xi[q]);
      } else {
        dr[q] = s ? next_digit(Xr[q]) : static_cast<int>(Xr[q]);
        di[q] = s ? next_digit(Xi[q]) : static_cast<int>(Xi[q]);
      }
    }
    __half* o = outz + s * plane;
    if (p.side == 0) {
      store_digits<PER, false>(o + r * p.kpad + l, dr);
      store_digits<PER, false>(o + r * p.kpad + K + l, di);
    } else {
      const long long row0 = 2LL * r, row1 = 2LL * r + 1;
      store_digits<PER, false>(o + row0 * p.kpad + l, dr);
      store_digits<PER, true>(o + row0 * p.kpad + K + l, di);
      store_digits<PER, false>(o + row1 * p.kpad + l, di);
      store_digits<PER, false>(o + row1 * p.kpad + K + l, dr);
    }
  }
}

// The same digits for a compile-time slice count SF (nbits = 8 SF - 1, 64-bit images), with
// no dependent chain per digit.  With C = 128 (1 + 256 + ... + 256^(SF-2)), Y = X + C holds
// the balanced digits d_s + 128 of the SF - 1 lower places as its low bytes and the top digit
// as Y >> 8 (SF - 1): X = sum_s d_s 256^s with every lower d_s in [-128, 127], so adding 128
// at each lower place lifts it into [0, 255] without carries, and base-256 digits are unique.
// Plane SF - 1 - s takes byte s of Y.  Two elements' bytes go into the halves of one word,
// offset by 0x6580 = (bit pattern of 1536 in binary16) - 128, which makes each half the bit
// pattern of 1536 + d (the binade [1024, 2048) has unit spacing); one packed subtraction of
// 1536 leaves d, and subtracting the word from 1536 leaves -d, both exact (+0 for d = 0, as
// the int -> half conversion gives).  The top digit (|d| <= 128) takes the offset 0x6600.
__host__ __device__ constexpr long long digit_bias(int S) {
  long long c = 0;
  for (int s = 0; s < S - 1; ++s) c = c * 256 + 128;
  return c;
}

struct Y64 { uint32_t lo, hi; };

// biased binary16 pair (bit patterns of 1536 + d) of plane `s` for two elements
template <int SF>
__device__ __forceinline__ uint32_t biased_pair(int s, Y64 a, Y64 b) {
  if (s > 0) {
    const int k = SF - 1 - s;                               // byte of Y, 0 .. SF - 2
    const uint32_t wa = k < 4 ? a.lo : a.hi, wb = k < 4 ? b.lo : b.hi;
    const uint32_t kk = static_cast<uint32_t>(k & 3);
    const uint32_t w = __byte_perm(wa, wb, kk | ((kk + 4u) << 8));
    return (w & 0x00FF00FFu) + 0x65806580u;
  }
  constexpr int sh = 8 * (SF - 1);
  const long long ya = static_cast<long long>((static_cast<unsigned long long>(a.hi) << 32) | a.lo);
  const long long yb = static_cast<long long>((static_cast<unsigned long long>(b.hi) << 32) | b.lo);
  const uint32_t ta = static_cast<uint32_t>(static_cast<int>(ya >> sh) + 0x6600);
  const uint32_t tb = static_cast<uint32_t>(static_cast<int>(yb >> sh) + 0x6600);
  return __byte_perm(ta, tb, 0x5410);
}

__device__ __forceinline__ uint32_t half2_bits(__half2 h) {
  return static_cast<uint32_t>(__half_as_ushort(__low2half(h))) |
         (static_cast<uint32_t>(__half_as_ushort(__high2half(h))) << 16);
}
__device__ __forceinline__ __half2 bits_half2(uint32_t w) {
  return __halves2half2(__ushort_as_half(static_cast<unsigned short>(w & 0xFFFFu)),
                        __ushort_as_half(static_cast<unsigned short>(w >> 16)));
}
// d (NEG: -d) of both halves of a biased pair
template <bool NEG>
__device__ __forceinline__ uint32_t pair_digits(uint32_t biased) {
  const __half2 k1536 = __half2half2(__ushort_as_half(0x6600));
  return half2_bits(NEG ? __hsub2(k1536, bits_half2(biased)) : __hsub2(bits_half2(biased), k1536));
}

template <int NW>
__device__ __forceinline__ void store_words(__half* dst, const uint32_t (&w)[NW]) {
  if constexpr (NW == 4) *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  else if constexpr (NW == 2) *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
  else *reinterpret_cast<uint32_t*>(dst) = w[0];
}

template <int PER, int SF>
__device__ __forceinline__ void split_run_fixed(const SplitParams& p, const double2* v, int e, int r, int l, int K,
                                                __half* outz, long long plane) {
  static_assert(PER >= 2 && PER % 2 == 0, "pairs of elements");
  constexpr long long C = digit_bias(SF);
  constexpr int NW = PER / 2;
  Y64 yr[PER], yi[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const unsigned long long a = static_cast<unsigned long long>(integer_image64(v[q].x, e, 8 * SF - 1) + C);
    const unsigned long long b = static_cast<unsigned long long>(integer_image64(v[q].y, e, 8 * SF - 1) + C);
    yr[q] = Y64{static_cast<uint32_t>(a), static_cast<uint32_t>(a >> 32)};
    yi[q] = Y64{static_cast<uint32_t>(b), static_cast<uint32_t>(b >> 32)};
  }
#pragma unroll
  for (int s = SF - 1; s >= 0; --s) {
    uint32_t br[NW], bi[NW], dr[NW], di[NW];
#pragma unroll
    for (int h = 0; h < NW; ++h) {
      br[h] = biased_pair<SF>(s, yr[2 * h], yr[2 * h + 1]);
      bi[h] = biased_pair<SF>(s, yi[2 * h], yi[2 * h + 1]);
      dr[h] = pair_digits<false>(br[h]);
      di[h] = pair_digits<false>(bi[h]);
    }
    __half* o = outz + s * plane;
    if (p.side == 0) {
      store_words<NW>(o + static_cast<long long>(r) * p.kpad + l, dr);
      store_words<NW>(o + static_cast<long long>(r) * p.kpad + K + l, di);
    } else {
      uint32_t ni[NW];
#pragma unroll
      for (int h = 0; h < NW; ++h) ni[h] = pair_digits<true>(bi[h]);
      const long long row0 = 2LL * r, row1 = 2LL * r + 1;
      store_words<NW>(o + row0 * p.kpad + l, dr);
      store_words<NW>(o + row0 * p.kpad + K + l, ni);
      store_words<NW>(o + row1 * p.kpad + l, di);
      store_words<NW>(o + row1 * p.kpad + K + l, dr);
    }
  }
}

// Both operands of one emulated GEMM in one launch: blockIdx.z selects the side.  VEC: the
// widest digit run stored as one vector (8 in general; 2 for K <= 16, where the runs are 2 wide
// and the smaller register footprint keeps more CTAs resident).  W64: 64-bit integer images
// (S <= 7).  Rows of at most SPLIT_TK elements (every panel operand of the block LU) are read
// from global memory once: the tile is loaded, the row maxima are taken from it, then the
// digits; longer rows take a scan pass and then the tiles one by one.
template <int VEC, bool W64, int SF = 0>
__global__ void __launch_bounds__(SPLIT_THREADS, VEC == 2 ? (W64 ? 5 : 4) : (W64 ? 4 : 2))
split_kernel(const SplitPair pp) {
  static_assert(SF == 0 || (W64 && VEC == 8), "compile-time slice counts: 64-bit images, 8-wide runs");
  if (static_cast<int>(blockIdx.z) >= pp.nsides) return;
  const SplitParams& p = pp.s[blockIdx.z];
  const int z = blockIdx.y;
  const bool single = p.X == nullptr;
  const int R = single ? p.rows1 : p.rows[z];
  const int K = single ? p.k1 : p.kdim[z];
  // K-parallel: CTA x = row block x / kgroups, the kg-th share of its K tiles
  const int kgs = p.kgroups > 1 ? p.kgroups : 1;
  const int kg = static_cast<int>(blockIdx.x) % kgs;
  const int r0 = (static_cast<int>(blockIdx.x) / kgs) * SPLIT_ROWS;
  if (r0 >= R) return;
  const double2* __restrict__ P = single ? p.X1 + z * p.zstride1 : p.X[z];
  const long long ld = single ? p.ld1 : p.ld[z];
  const int tid = threadIdx.x;
  const bool kpar = kgs > 1 && K > SPLIT_TK;
  const bool one_tile = K <= SPLIT_TK;

  __shared__ unsigned long long rowmax[SPLIT_ROWS];
  __shared__ int rowexp[SPLIT_ROWS];
  __shared__ int rowbad[SPLIT_ROWS];
  __shared__ double2 tile[SPLIT_ROWS][SPLIT_TK + 1];
  __shared__ int bad;
  if (tid < SPLIT_ROWS) { rowmax[tid] = 0ull; rowbad[tid] = 0; }
  if (tid == 0) bad = 0;
  __syncthreads();

  // tile width along K: 64, or K rounded up to 8 for short rows (so no thread idles on padding)
  const int TK = K >= SPLIT_TK ? SPLIT_TK : ((K + 7) & ~7);
  const int per = TK / 8;                      // consecutive l per thread
  // a 32 x TK tile starting at column lt (coalesced along the stored contiguous direction);
  // non-finite scalars are flagged (their row's exponent becomes 0, as a non-finite maximum
  // gives) and split as zero
  auto load_tile = [&](int lt) {
    // all of a thread's loads are issued before any is used, so their latencies overlap (tiles
    // are at most 16 wide in the VEC = 2 instance, which serves K <= 16 only)
    constexpr int NPT = SPLIT_ROWS * (VEC == 2 ? 16 : SPLIT_TK) / SPLIT_THREADS;
    longlong2 v[NPT];
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
      const int idx = tid + u * SPLIT_THREADS;
      int rl, ll;
      if (!p.trans) { rl = idx % SPLIT_ROWS; ll = idx / SPLIT_ROWS; }
      else          { ll = idx % TK;         rl = idx / TK; }
      const int r = r0 + rl, l = lt + ll;
      v[u] = make_longlong2(0, 0);
      if (idx < SPLIT_ROWS * TK && r < R && l < K)
        v[u] = reinterpret_cast<const longlong2*>(P)[p.trans ? l + r * ld : r + l * ld];
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
      const int idx = tid + u * SPLIT_THREADS;
      if (idx >= SPLIT_ROWS * TK) break;
      int rl, ll;
      if (!p.trans) { rl = idx % SPLIT_ROWS; ll = idx / SPLIT_ROWS; }
      else          { ll = idx % TK;         rl = idx / TK; }
      // integer operations on the bit patterns only (binary64 compares and negations would
      // occupy this GPU's scarce FP64 pipe)
      longlong2 w = v[u];
      if (p.conj) w.y ^= static_cast<long long>(0x8000000000000000ull);
      const bool fx = (w.x & 0x7FF0000000000000ll) == 0x7FF0000000000000ll;
      const bool fy = (w.y & 0x7FF0000000000000ll) == 0x7FF0000000000000ll;
      if (fx || fy) {
        bad = 1;
        rowbad[rl] = 1;
        if (fx) w.x = 0;
        if (fy) w.y = 0;
      }
      tile[rl][ll] = make_double2(__longlong_as_double(w.x), __longlong_as_double(w.y));
    }
  };

  if (kpar) {
    // row maxima taken by the pre-pass over all of K (a non-finite maximum flags the row)
    if (tid < SPLIT_ROWS && r0 + tid < R) {
      rowmax[tid] = p.gmax[z * p.exp_stride + r0 + tid];
      if (rowmax[tid] >= 0x7FF0000000000000ull) bad = 1;
    }
  } else if (one_tile) {
    load_tile(0);
    __syncthreads();
    // row maxima from the tile: 8 threads per row, combined by shuffles
    const int rl = tid >> 3, cg = tid & 7;
    unsigned long long mx = 0ull;
    for (int l = cg; l < K; l += 8) {
      const double2 v = tile[rl][l];
      const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v.x)) & 0x7FFFFFFFFFFFFFFFull;
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v.y)) & 0x7FFFFFFFFFFFFFFFull;
      mx = max(mx, max(a, b));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (cg == 0) rowmax[rl] = rowbad[rl] ? 0x7FF0000000000000ull : mx;
  } else {
    // ---- scan pass: row maxima
    int rl, l0, lstep;
    if (!p.trans) { rl = tid % SPLIT_ROWS; l0 = tid / SPLIT_ROWS; lstep = SPLIT_THREADS / SPLIT_ROWS; }
    else          { rl = tid / 8;          l0 = tid % 8;          lstep = 8; }
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
  if (tid < SPLIT_ROWS) {
    const unsigned long long a = rowmax[tid];
    const int e = (a >= 0x7FF0000000000000ull) ? 0 : frexp_exponent_from_bits(a);
    rowexp[tid] = e;
    if (r0 + tid < R && kg == 0) p.exps[z * p.exp_stride + r0 + tid] = e;
  }
  __syncthreads();

  // ---- digits, tile by tile along K
  const int S = p.S;
  const long long plane = p.out_rows * p.kpad;
  __half* outz = p.out + static_cast<long long>(z) * S * plane;
  const bool dbg = (p.dbg_digits != nullptr) && z == 0;
  const long long dplane = p.out_rows * 2LL * K;
  int lt_begin = 0, lt_end = K;
  if (kpar) {
    const int ntk = (K + TK - 1) / TK, per_g = (ntk + kgs - 1) / kgs;
    lt_begin = kg * per_g * TK;
    lt_end = min(K, (kg + 1) * per_g * TK);
  }
  for (int lt = lt_begin; lt < lt_end; lt += TK) {
    if (!one_tile) {
      load_tile(lt);
      __syncthreads();
    }
    // each thread: one row, 8 consecutive l
    {
      const int rl = tid / 8;
      const int lg = (tid % 8) * per;
      const int r = r0 + rl;
      const int l0 = lt + lg;
      // vector stores when this thread's run is whole and aligned (and no debug copy)
      const bool vec = !dbg && ((VEC >= 8 && per == 8) || (VEC >= 4 && per == 4) || per == 2) && K % per == 0 &&
                       l0 + per <= K;
      if (r < R && vec) {
        const int e = rowexp[rl];
        if constexpr (SF > 0) {
          if (per == 8) split_run_fixed<8, SF>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
          else if (per == 4) split_run_fixed<4, SF>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
          else split_run_fixed<2, SF>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
        } else if constexpr (VEC >= 8) {
          if (per == 8) split_run<8, W64>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
          else if (per == 4) split_run<4, W64>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
          else split_run<2, W64>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
        } else {
          split_run<2, W64>(p, &tile[rl][lg], e, r, l0, K, outz, plane);
        }
      } else if (r < R) {
        const int e = rowexp[rl];
        for (int q = 0; q < per; ++q) {
          const int l = lt + lg + q;
          if (l >= K) break;
          const double2 v = tile[rl][lg + q];
          __int128 Xr = integer_image(v.x, e, p.nbits);
          __int128 Xi = integer_image(v.y, e, p.nbits);
          // digits from the least significant (plane S-1) to the most significant (plane 0)
          for (int s = S - 1; s >= 0; --s) {
            const int dr = s ? next_digit(Xr) : static_cast<int>(Xr);
            const int di = s ? next_digit(Xi) : static_cast<int>(Xi);
            __half* o = outz + s * plane;
            if (p.side == 0) {
              o[r * p.kpad + l] = __int2half_rn(dr);
              o[r * p.kpad + K + l] = __int2half_rn(di);
              if (dbg) {
                p.dbg_digits[s * dplane + r * 2LL * K + l] = static_cast<int16_t>(dr);
                p.dbg_digits[s * dplane + r * 2LL * K + K + l] = static_cast<int16_t>(di);
              }
            } else {
              const long long row0 = 2LL * r, row1 = 2LL * r + 1;
              o[row0 * p.kpad + l] = __int2half_rn(dr);
              o[row0 * p.kpad + K + l] = __int2half_rn(-di);
              o[row1 * p.kpad + l] = __int2half_rn(di);
              o[row1 * p.kpad + K + l] = __int2half_rn(dr);
              if (dbg) {
                p.dbg_digits[s * dplane + row0 * 2LL * K + l] = static_cast<int16_t>(dr);
                p.dbg_digits[s * dplane + row0 * 2LL * K + K + l] = static_cast<int16_t>(-di);
                p.dbg_digits[s * dplane + row1 * 2LL * K + l] = static_cast<int16_t>(di);
                p.dbg_digits[s * dplane + row1 * 2LL * K + K + l] = static_cast<int16_t>(dr);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // zero the K padding [2K, kpad) of the rows this CTA owns (one CTA of a row block)
  const int pad = static_cast<int>(p.kpad) - 2 * K;
  if (pad > 0 && kg == kgs - 1) {
    const int rows_out = p.side == 0 ? 1 : 2;
    const int nr = min(SPLIT_ROWS, R - r0) * rows_out;
    for (int idx = tid; idx < S * nr * pad; idx += SPLIT_THREADS) {
      const int c = idx % pad;
      const int rr = (idx / pad) % nr;
      const int s = idx / (pad * nr);
      outz[s * plane + (static_cast<long long>(r0) * rows_out + rr) * p.kpad + 2 * K + c] = __float2half(0.0f);
    }
  }
}

// Row maxima for the K-parallel split: CTA x covers 32 rows (x / nseg) and K segment x % nseg
// of SPLIT_KSEG elements; each row's largest |Re|, |Im| bit pattern (non-finite values compare
// above every finite one) reaches gmax by one 64-bit atomicMax per row and CTA.
constexpr int SPLIT_KSEG = 512;
__global__ void __launch_bounds__(SPLIT_THREADS) split_rowmax_kernel(const SplitPair pp, int nseg) {
  if (static_cast<int>(blockIdx.z) >= pp.nsides) return;
  const SplitParams& p = pp.s[blockIdx.z];
  if (!p.gmax) return;
  const int z = blockIdx.y;
  const bool single = p.X == nullptr;
  const int R = single ? p.rows1 : p.rows[z];
  const int K = single ? p.k1 : p.kdim[z];
  const int r0 = (static_cast<int>(blockIdx.x) / nseg) * SPLIT_ROWS;
  const int l_lo = (static_cast<int>(blockIdx.x) % nseg) * SPLIT_KSEG;
  if (r0 >= R || l_lo >= K) return;
  const int l_hi = min(K, l_lo + SPLIT_KSEG);
  const double2* __restrict__ P = single ? p.X1 + z * p.zstride1 : p.X[z];
  const long long ld = single ? p.ld1 : p.ld[z];
  __shared__ unsigned long long mx_s[SPLIT_ROWS];
  const int tid = threadIdx.x;
  if (tid < SPLIT_ROWS) mx_s[tid] = 0ull;
  __syncthreads();
  int rl, l0, lstep;
  if (!p.trans) { rl = tid % SPLIT_ROWS; l0 = tid / SPLIT_ROWS; lstep = SPLIT_THREADS / SPLIT_ROWS; }
  else          { rl = tid / 8;          l0 = tid % 8;          lstep = 8; }
  const int r = r0 + rl;
  if (r < R) {
    unsigned long long mx = 0ull;
    for (int l = l_lo + l0; l < l_hi; l += lstep) {
      const double2 v = p.trans ? P[l + r * ld] : P[r + l * ld];
      const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v.x)) & 0x7FFFFFFFFFFFFFFFull;
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v.y)) & 0x7FFFFFFFFFFFFFFFull;
      mx = max(mx, max(a, b));
    }
    atomicMax(&mx_s[rl], mx);
  }
  __syncthreads();
  if (tid < SPLIT_ROWS && r0 + tid < R) atomicMax(&p.gmax[z * p.exp_stride + r0 + tid], mx_s[tid]);
}

void launch_split(const SplitParams& a, int rows_a, const SplitParams* b, int rows_b, int kmax, int batch,
                  cudaStream_t st) {
  SplitPair pp;
  pp.s[0] = a;
  pp.nsides = b ? 2 : 1;
  if (b) pp.s[1] = *b;
  const int rows = std::max(rows_a, b ? rows_b : 0);
  const int rblocks = (rows + SPLIT_ROWS - 1) / SPLIT_ROWS;
  // few row blocks and rows longer than one tile: share each row block's K tiles among kgroups
  // CTAs, after a pre-pass that takes the row maxima over K segments
  int kgroups = 1;
  const bool can_kpar = pp.s[0].gmax && (pp.nsides < 2 || pp.s[1].gmax);
  if (can_kpar && kmax > SPLIT_TK) {
    const long long ctas = static_cast<long long>(rblocks) * batch * pp.nsides;
    const int sms = gpu_sm_count();
    if (ctas < sms) {
      const int ntk = (kmax + SPLIT_TK - 1) / SPLIT_TK;
      kgroups = static_cast<int>(std::min<long long>(ntk, std::max<long long>(1, (2LL * sms) / ctas)));
    }
  }
  for (int sd = 0; sd < pp.nsides; ++sd) pp.s[sd].kgroups = kgroups;
  if (kgroups > 1) {
    const int nseg = (kmax + SPLIT_KSEG - 1) / SPLIT_KSEG;
    for (int sd = 0; sd < pp.nsides; ++sd)
      cudaMemsetAsync(pp.s[sd].gmax, 0, sizeof(unsigned long long) * pp.s[sd].exp_stride * batch, st);
    split_rowmax_kernel<<<dim3(rblocks * nseg, batch, pp.nsides), SPLIT_THREADS, 0, st>>>(pp, nseg);
    record_launch();
  }
  dim3 grid(rblocks * kgroups, batch, pp.nsides);
  const bool w64 = pp.s[0].nbits <= 62 && (pp.nsides < 2 || pp.s[1].nbits <= 62);
  if (kmax <= 16) {
    if (w64) split_kernel<2, true><<<grid, SPLIT_THREADS, 0, st>>>(pp);
    else split_kernel<2, false><<<grid, SPLIT_THREADS, 0, st>>>(pp);
  } else {
    // compile-time slice counts for the common S = 7 and S = 5 (nbits = 8 S - 1 on every side)
    int sf = 0;
    for (int S : {7, 5}) {
      bool all = true;
      for (int sd = 0; sd < pp.nsides; ++sd) all = all && pp.s[sd].S == S && pp.s[sd].nbits == 8 * S - 1;
      if (all) { sf = S; break; }
    }
    if (sf == 7) split_kernel<8, true, 7><<<grid, SPLIT_THREADS, 0, st>>>(pp);
    else if (sf == 5) split_kernel<8, true, 5><<<grid, SPLIT_THREADS, 0, st>>>(pp);
    else if (w64) split_kernel<8, true><<<grid, SPLIT_THREADS, 0, st>>>(pp);
    else split_kernel<8, false><<<grid, SPLIT_THREADS, 0, st>>>(pp);
  }
  record_launch();
}

}  // namespace ozk
