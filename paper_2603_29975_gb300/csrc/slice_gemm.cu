// Slice-pair GEMM on the sm_103a tensor cores with the fused reconstruction epilogue
// (paper Sec. 2.2: low-precision products of slice pairs, accumulated in higher precision).
//
// Operands are the fp16 digit planes written by split.cu: A [batch][S][rowsA][kpad] and B
// [batch][S][rowsB][kpad] (K-major).  One CTA computes a 128 x BN tile of the stacked real
// product (m x 2n) for every slice pair at once:
//
//   * warp 0 (one lane) streams K-blocks of 16 with TMA: one 3-D box of S slices of A
//     (128 rows) and one of B (BN rows) per pipeline stage, 32-byte swizzle;
//   * warp 1 (one lane) issues tcgen05.mma kind::f16 for every pair (s, t) of the pair set,
//     accumulating pair products of the same weight class g = s + t into one FP32 TMEM
//     accumulator per group (G groups x BN columns of the 512); after a chunk's first K-block
//     the partners of each A slice share one MMA over the stacked B slices;
//   * warps 2..17 drain the accumulators.  Every product of two digits is an integer of
//     magnitude <= 2^14 and each accumulator receives at most 1024 of them per "exactness
//     chunk" of K, so every FP32 value is an exact integer <= 2^24.  The epilogue converts
//     it to int32 and adds it, shifted by its group weight 8 (g_max - g) bits, into a 64-bit
//     (when the exact sum fits) or 128-bit integer per output element; after the last chunk
//     that integer times 2^(e_i + f_j + c) is rounded once to binary64 (the int64 -> binary64
//     conversion of the exact sum, or of a sticky-jammed 64-bit image of the 128-bit sum),
//     then stored (C = Z), or subtracted from C (LU update), or combined with alpha/beta.
// No floating-point instruction touches the products' sums before that one rounding; the
// only binary64 arithmetic after it is the subtraction / alpha-beta combination per element.
#include <algorithm>

#include "ozk_params.cuh"

namespace ozk {

constexpr int GEMM_BM = 128;
constexpr int GEMM_EPI_WARPS = 16;
// warpgroup 0 (warps 0..3): TMA producer (warp 0), MMA issuer (warp 1), two idle warps; it
// hands registers to the four epilogue warpgroups (setmaxnreg), whose exact 128-bit sums need
// more than the 96 registers a thread of a 20-warp CTA starts with
constexpr int GEMM_CTRL_WARPS = 4;
constexpr int GEMM_THREADS = (GEMM_CTRL_WARPS + GEMM_EPI_WARPS) * 32;
constexpr int GEMM_CTRL_REGS = 64, GEMM_EPI_REGS = 104;


// RN-even of (H 2^S8 + L) 2^E for int64 H, L with |H| < 2^56 and |L| < 2^(S8 + 30), S8 <= 32,
// through the int64 -> binary64 conversion (RN-even to 53 bits) of one 64-bit integer:
// H' = H + floor(L / 2^S8) and Ll = L mod 2^S8 give the exact T = H' 2^S8 + Ll.  When T fits in
// 62 bits it is converted as it is; otherwise T is shifted right by sh <= S8 bits (so that
// 2^61 <= |T'| < 2^62) and the dropped bits of Ll are jammed into bit 0 of T' as a sticky bit:
// T' then has more than two bits below the rounding position and no midpoint on its odd bit,
// so its RN-even is that of T / 2^sh (round-to-odd argument).  The scaling by 2^(E + sh) is an
// exponent-field addition while the result stays normal; other results take the general
// 128-bit routine.
template <int S8>
__device__ __forceinline__ double round_hl_jam(long long H, long long L, int E) {
  long long Hp = H, Ll = 0;
  if constexpr (S8 > 0) {
    Hp = H + (L >> S8);
    Ll = L & ((1ll << S8) - 1);
  }
  const unsigned long long mag = static_cast<unsigned long long>(Hp < 0 ? -Hp : Hp);
  const int b = 64 - __clzll(mag);                        // bit length of |H'|
  const int sh = max(0, b + S8 - 62);
  long long T;
  if constexpr (S8 > 0) {
    T = static_cast<long long>(static_cast<unsigned long long>(Hp) << (S8 - sh)) + (Ll >> sh);
    T |= (Ll & ((1ll << sh) - 1)) != 0 ? 1ll : 0ll;
  } else {
    T = Hp;
  }
  const double d = __ll2double_rn(T);
  const long long bits = __double_as_longlong(d);
  const int ed = static_cast<int>((bits >> 52) & 0x7FF);
  if (ed == 0) return d;                                    // T = 0
  const int Et = E + sh;
  if (ed + Et < 1 || ed + Et > 2046) {
    const __int128 v = (static_cast<__int128>(H) << S8) + static_cast<__int128>(L);
    return round_scaled_dev(v, E);
  }
  return __longlong_as_double(bits + (static_cast<long long>(Et) << 52));
}

// Exact FP32 integer accumulator value -> int32.  "magic": |v| < 2^22, one FP32 add puts the
// integer in the low mantissa bits; otherwise the hardware conversion (exact for |v| <= 2^24).
__device__ __forceinline__ int acc_to_int(uint32_t bits, bool magic) {
  const float x = __uint_as_float(bits);
  return magic ? (__float_as_int(x + 12582912.0f) - 0x4B400000) : __float2int_rn(x);
}

// V[j] += v_j w for 8 exact FP32 accumulators of one group.  MAGIC (uniform over the warp):
// the group's accumulators stay within 2^22 in magnitude, so one FP32 add and a reinterpret
// convert them (x + 1.5 2^23 lies in [2^23, 2^24], where every integer is representable);
// otherwise the hardware conversion.  The branch keeps the conversion unit out of the first
// case.
__device__ __forceinline__ void fold8(long long* V, const uint32_t (&v)[8], long long w, bool magic) {
  if (magic) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      V[j] += static_cast<long long>(__float_as_int(__uint_as_float(v[j]) + 12582912.0f) - 0x4B400000) * w;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) V[j] += static_cast<long long>(__float2int_rn(__uint_as_float(v[j]))) * w;
  }
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t& a, uint32_t& b) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr));
}

// Compile-time slice-pair schedule (a chunk's first K-block): pairs (s, t) in order of their
// group g = s + t, the first pair of each group flagged.  The MMA issuer walks it fully
// unrolled, so one MMA costs two 32-bit descriptor additions and the tcgen05.mma itself.
__device__ __forceinline__ void mma_f16_lo(uint32_t d_tmem, uint32_t a_lo, uint32_t b_lo, uint32_t hi, uint32_t idesc,
                                           uint32_t accumulate) {
  const uint64_t ad = (static_cast<uint64_t>(hi) << 32) | a_lo;
  const uint64_t bd = (static_cast<uint64_t>(hi) << 32) | b_lo;
  mma_f16(d_tmem, ad, bd, idesc, accumulate);
}

// One K-block of MMAs for every pair.  FIRST: first K-block of an exactness chunk -- the first
// pair of each group overwrites its accumulator (after the epilogue released it, when
// `wait_release`); returns false if a wait gave up.
template <int S, bool FULLSET, int BN, bool FIRST>
__device__ __forceinline__ bool issue_kblock(uint32_t tmem, uint32_t a_lo, uint32_t b_lo, uint32_t hi, uint32_t idesc,
                                             uint64_t* acc_empty, uint32_t rel_parity, bool wait_release, int* status,
                                             volatile int* abort_flag) {
  constexpr int GMAX = FULLSET ? 2 * S : S + 1;
#pragma unroll
  for (int g = 2; g <= GMAX; ++g) {
    bool first = true;
#pragma unroll
    for (int s = 1; s <= S; ++s) {
      const int t = g - s;
      if (t < 1 || t > S) continue;
      if (FIRST && first && wait_release) {
        if (!mbar_wait(&acc_empty[g - 2], rel_parity, status, abort_flag)) return false;
        tc_fence_after();
      }
      mma_f16_lo(tmem + (g - 2) * BN, a_lo + (s - 1) * (GEMM_BM * 32 / 16), b_lo + (t - 1) * (BN * 32 / 16), hi, idesc,
                 (FIRST && first) ? 0u : 1u);
      first = false;
    }
  }
  return true;
}

// A later K-block of a chunk: every accumulator is live, so the partners of A slice s can share
// one A read.  The B slices sit back to back in shared memory (slice t at row (t - 1) BN) and
// group g = s + t at TMEM column (g - 2) BN, so A_s x [B_1 .. B_nt]^T is a single MMA of
// N = nt BN landing on the columns of groups s + 1 .. s + nt (split at N = 256).  Same products,
// same accumulators as the pair-by-pair order; a third of the A traffic out of shared memory.
template <int S, bool FULLSET, int BN>
__device__ __forceinline__ void issue_kblock_stacked(uint32_t tmem, uint32_t a_lo, uint32_t b_lo, uint32_t hi) {
#pragma unroll
  for (int s = 1; s <= S; ++s) {
    constexpr int NMAX = 256;
    const int ncols = (FULLSET ? S : S + 1 - s) * BN;
#pragma unroll
    for (int c0 = 0; c0 < ncols; c0 += NMAX) {
      const int n = ncols - c0 < NMAX ? ncols - c0 : NMAX;
      mma_f16_lo(tmem + (s - 1) * BN + c0, a_lo + (s - 1) * (GEMM_BM * 32 / 16), b_lo + c0 * (32 / 16), hi,
                 idesc_f16_f32(GEMM_BM, n), 1u);
    }
  }
}

// A chunk's first K-block with the triangular pair set: slice s = 1 pairs with every t = 1..S,
// so it is the first writer of every group g = 1 + t.  Once the epilogue has released all the
// accumulators of the previous chunk, A_1 x [B_1 .. B_S]^T overwrites every group in one
// stacked MMA (accumulate = 0) and the later A slices accumulate onto it, as in the later
// K-blocks: S MMAs (plus the N = 256 splits) instead of one per pair.
template <int S, int BN>
__device__ __forceinline__ bool issue_kblock_first_stacked(uint32_t tmem, uint32_t a_lo, uint32_t b_lo, uint32_t hi,
                                                           uint64_t* acc_empty, uint32_t rel_parity, bool wait_release,
                                                           int* status, volatile int* abort_flag) {
#pragma unroll
  for (int s = 1; s <= S; ++s) {
    constexpr int NMAX = 256;
    const int ncols = (S + 1 - s) * BN;
#pragma unroll
    for (int c0 = 0; c0 < ncols; c0 += NMAX) {
      const int n = ncols - c0 < NMAX ? ncols - c0 : NMAX;
      if (s == 1 && wait_release) {
        // the groups this MMA overwrites (TMEM columns [c0, c0 + n)): it starts as soon as the
        // epilogue has released them, while the later groups are still being drained
#pragma unroll
        for (int g = c0 / BN; g < (c0 + n) / BN; ++g)
          if (!mbar_wait(&acc_empty[g], rel_parity, status, abort_flag)) return false;
        tc_fence_after();
      }
      mma_f16_lo(tmem + (s - 1) * BN + c0, a_lo + (s - 1) * (GEMM_BM * 32 / 16), b_lo + c0 * (32 / 16), hi,
                 idesc_f16_f32(GEMM_BM, n), s > 1 ? 1u : 0u);
    }
  }
  return true;
}

template <int S, bool FULLSET, int BN>
__device__ __forceinline__ bool issue_kblock_any(bool firstkb, uint32_t tmem, uint32_t a_lo, uint32_t b_lo, uint32_t hi,
                                                 uint32_t idesc, uint64_t* acc_empty, uint32_t rel_parity,
                                                 bool wait_release, int* status, volatile int* abort_flag) {
  if (firstkb) {
    if constexpr (!FULLSET)
      return issue_kblock_first_stacked<S, BN>(tmem, a_lo, b_lo, hi, acc_empty, rel_parity, wait_release, status,
                                               abort_flag);
    return issue_kblock<S, FULLSET, BN, true>(tmem, a_lo, b_lo, hi, idesc, acc_empty, rel_parity, wait_release, status,
                                              abort_flag);
  }
  issue_kblock_stacked<S, FULLSET, BN>(tmem, a_lo, b_lo, hi);
  return true;
}

// Runtime schedule (S > 8, or S > 4 with the full pair set: the 32-column tiles).
template <int BN>
__device__ __forceinline__ bool issue_runtime(const GemmParams& p, bool firstkb, uint32_t tmem, uint32_t a_lo,
                                              uint32_t b_lo, uint32_t hi, uint32_t idesc, uint64_t* acc_empty,
                                              uint32_t rel_parity, bool wait_release, volatile int* abort_flag) {
  for (int pi = 0; pi < p.npairs; ++pi) {
    const uint32_t s = p.ps[pi], t = p.pt[pi], g = p.pg[pi];
    const bool first = firstkb && p.pfirst[pi];
    if (first && wait_release) {
      if (!mbar_wait(&acc_empty[g], rel_parity, p.status, abort_flag)) return false;
      tc_fence_after();
    }
    mma_f16_lo(tmem + g * BN, a_lo + s * (GEMM_BM * 32 / 16), b_lo + t * (BN * 32 / 16), hi, idesc, first ? 0u : 1u);
  }
  return true;
}

template <int BN>
__device__ __forceinline__ bool issue_dispatch(int S, bool fullset, bool firstkb, uint32_t tmem, uint32_t a_lo,
                                               uint32_t b_lo, uint32_t hi, uint32_t idesc, uint64_t* acc_empty,
                                               uint32_t rel_parity, bool wait_release, int* status,
                                               volatile int* abort_flag) {
#define OZK_ISSUE(SS, FF) return issue_kblock_any<SS, FF, BN>(firstkb, tmem, a_lo, b_lo, hi, idesc, acc_empty, rel_parity, wait_release, status, abort_flag)
  if constexpr (BN == 64) {
    if (!fullset) {
      switch (S) { case 1: OZK_ISSUE(1, false); case 2: OZK_ISSUE(2, false); case 3: OZK_ISSUE(3, false);
                   case 4: OZK_ISSUE(4, false); case 5: OZK_ISSUE(5, false); case 6: OZK_ISSUE(6, false);
                   case 7: OZK_ISSUE(7, false); default: OZK_ISSUE(8, false); }
    } else {
      switch (S) { case 1: OZK_ISSUE(1, true); case 2: OZK_ISSUE(2, true); case 3: OZK_ISSUE(3, true);
                   default: OZK_ISSUE(4, true); }
    }
  } else {
    // 32-column tiles: the triangular sets of S = 9 (the selector's largest regular choice)
    // and S = 10 (its fallback); the caller sends every other case to the runtime schedule
    if (S == 9) OZK_ISSUE(9, false);
    OZK_ISSUE(10, false);
  }
#undef OZK_ISSUE
}

// the compile-time schedules of issue_dispatch cover this launch
template <int BN>
__device__ __forceinline__ bool dispatch_covers(const GemmParams& p, int S) {
  if (p.diag_pairs) return false;
  if constexpr (BN == 64) return true;
  return !p.fullset && (S == 9 || S == 10);
}

// Tiles of one problem of a batched GEMM (m rows, n2 stacked columns) with a skip box
// [0, km) x [0, kn) (rows, complex columns) whose outputs are neither computed nor written: the
// part beside the box, rows [0, km) x stacked columns [2 kn, n2), in ku x xu tiles of a grid
// that starts at row 0 and stacked column 2 kn (the last tile row clipped at row km, mu), then
// the part below it, rows [km, m) x all columns, in nl x ntx tiles of a grid that starts at row
// km (m0l).  Each part's grid starts at the box edge, so a strip of one tile's width beside or
// below the box takes one tile row or column, not two.  Without a box (km or kn zero) the whole
// grid is the second part.
struct BoxTiles { int ku, xu, mu, n0u, nl, ntx, m0l; };
__host__ __device__ __forceinline__ BoxTiles box_tiles(int m, int n2, int km, int kn, int BN) {
  BoxTiles b;
  b.ntx = (n2 + BN - 1) / BN;
  if (km > 0 && kn > 0) {
    b.mu = km < m ? km : m;
    b.ku = (b.mu + GEMM_BM - 1) / GEMM_BM;
    b.n0u = 2 * kn;
    b.xu = n2 > b.n0u ? (n2 - b.n0u + BN - 1) / BN : 0;
    b.m0l = km;
    b.nl = m > km ? (m - km + GEMM_BM - 1) / GEMM_BM : 0;
  } else {
    b.mu = 0; b.ku = 0; b.n0u = 0; b.xu = 0; b.m0l = 0;
    b.nl = (m + GEMM_BM - 1) / GEMM_BM;
  }
  return b;
}

struct EpiCtx {
  int row, z, m_z, n2_z, n0, c0, skip_n, er;
  int sp;                // split-K: the unit's K slice (its partial sums go to p.part)
  int grow;              // row of the output matrix (the diagonal test of EPI_IMINUS)
  int jlim;              // complex columns of the output row's matrix
  uint32_t tbase;
  double2* Cz;           // output row r is Cz[crow + column * ldc]
  long long crow, ldc;
  bool rowok;
};

// output matrix, row offset, matrix row, leading dimension and column count of tile row
// `row` of problem z; clears rowok for rows past their matrix
// (za, ra: the operand plane and first plane row of the problem; z, 0 without a remap table)
__device__ __forceinline__ void out_row(const GemmParams& p, bool single, int z, int row, int za, int ra, bool& rowok,
                                        double2*& Cz, long long& crow, int& grow, long long& ldc, int& jlim) {
  if (p.crow) {
    const int pr = ra + row;                                  // row of the operand plane
    const int as = pr / p.crow_b, rl = pr - as * p.crow_b;
    const int a = p.crow_perm ? (rowok ? p.crow_perm[as] : 0) : as;
    Cz = rowok ? p.crow[a] : nullptr;
    crow = static_cast<long long>(za) * p.crow_b + rl;
    grow = static_cast<int>(crow);
    if (p.crow_n) {
      const int na = rowok ? p.crow_n[a] : 0;
      if (crow >= na) rowok = false;
      ldc = na;
      jlim = na;
    } else {
      ldc = p.ldc1;
      jlim = 0x7FFFFFFF;
    }
  } else {
    Cz = single ? p.C1 : p.C[z];
    crow = row;
    grow = row;
    ldc = single ? p.ldc1 : p.ldc[z];
    jlim = 0x7FFFFFFF;
  }
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
}

__device__ __forceinline__ void prefetch_l2(const void* ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<uint64_t>(ptr)));
}

// Waits of the epilogue for the accumulators of one tile: its exactness chunks complete one
// after the other on acc_full (chunk counter cc, running over the CTA's tiles).
struct ChunkWait {
  uint64_t* acc_full;
  int nchunks;
  uint32_t* cc;
  int* status;
  volatile int* abort_flag;
  __device__ __forceinline__ bool next() {
    if (!mbar_wait(acc_full, *cc & 1, status, abort_flag)) return false;
    tc_fence_after();
    ++*cc;
    return true;
  }
};

// Release every group accumulator of every chunk of a tile without reading it (a warp with no
// output in the tile).
template <int G>
__device__ __forceinline__ bool release_unread(uint64_t* acc_empty, ChunkWait& cw, int lane) {
  for (int c = 0; c < cw.nchunks; ++c) {
    if (!cw.next()) return false;
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[gi]);
    }
  }
  return true;
}

// Epilogue of one 128 x 64 tile for G <= 8 groups (compile-time) over the tile's exactness
// chunks: the exact sum of the group values v_g (|v| <= 2^24 per chunk) is H 2^(8 NL) + L with
// H = the first NH = min(G, 4) groups and L = the rest, each accumulated over the chunks by
// 32 x 32 -> 64-bit multiply-adds with constant weights 2^24, 2^16, 2^8, 1 (|H|, |L| < 2^49 per
// chunk).  A thread owns one row and 16 stacked columns (8 complex).  Each group accumulator is
// released as soon as it is read, so the MMAs of the next chunk or tile start while the last
// chunk is rounded and written.  The 16 sums are rounded as soon as the drain ends (the two
// 64-bit halves of every sum die there), then all of the thread's C values are requested at
// once and combined.  Returns false if a wait gave up.
template <int G, bool KS = false>
__device__ __forceinline__ bool epilogue_fast(const GemmParams& p, const EpiCtx& x, uint64_t* acc_empty, bool magic,
                                              int lane, ChunkWait& cw) {
  constexpr int NH = G < 4 ? G : 4;
  constexpr int NL = G - NH;
  constexpr int S8 = 8 * NL;
  constexpr int BN = 64;
  const bool needC = p.mode == EPI_LU || p.mode == EPI_GENERAL;
  const int jc0 = (x.n0 + x.c0) / 2;                  // this thread's 8 complex columns
  const int jend = min(min(jc0 + 8, (x.n2_z + 1) / 2), x.jlim);
  const bool active = x.rowok && max(jc0, x.skip_n) < jend;
  if (!__any_sync(0xffffffffu, active)) return release_unread<G>(acc_empty, cw, lane);
  // phase A: drain -- fold every group of the 16 columns into H, L and release its
  // accumulator at once, chunk after chunk
  long long H[16], L[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { H[j] = 0; L[j] = 0; }
  for (int c = 0; c < cw.nchunks; ++c) {
    if (!cw.next()) return false;
    if (c == cw.nchunks - 1 && needC && active) {
      // C lines towards L2 now, consumed after the drain
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (jc0 + jj < jend) prefetch_l2(x.Cz + x.crow + (jc0 + jj) * x.ldc);
    }
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      uint32_t v[8], u[8];
      tmem_ld8(x.tbase + gi * BN, v);
      tmem_ld8(x.tbase + gi * BN + 8, u);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[gi]);         // group gi may be overwritten now
      const int w = gi < NH ? (1 << (8 * (NH - 1 - gi))) : (1 << (8 * (NL - 1 - (gi - NH))));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long a = static_cast<long long>(acc_to_int(v[j], magic)) * w;
        const long long b = static_cast<long long>(acc_to_int(u[j], magic)) * w;
        if (gi < NH) { H[j] += a; H[j + 8] += b; } else { L[j] += a; L[j + 8] += b; }
      }
    }
  }
  if constexpr (KS) {
    // split K: the exact 64-bit halves of this unit's partial sums, column-major (coalesced over
    // the warp's rows); finish_split adds the units and rounds once
    if (x.rowok) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = x.n0 + x.c0 + j;
        if (col < x.n2_z) p.part[(static_cast<long long>(x.sp) * x.n2_z + col) * p.m1 + x.row] = make_longlong2(H[j], L[j]);
      }
    }
    return true;
  }
  if (!active) return true;
  // the 16 roundings (column exponents from memory), then phase B: every C value of the
  // thread requested at once, combined and written
  double zz[16];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int jc = jc0 + jj;
    const int E = x.er + (jc < jend ? p.f[x.z * p.f_stride + jc] : 0);
    zz[2 * jj] = round_hl_jam<S8>(H[2 * jj], L[2 * jj], E);
    zz[2 * jj + 1] = round_hl_jam<S8>(H[2 * jj + 1], L[2 * jj + 1], E);
  }
  double2 cv[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int jc = jc0 + jj;
    cv[jj] = (needC && jc < jend && jc >= x.skip_n) ? x.Cz[x.crow + jc * x.ldc] : make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int jc = jc0 + jj;
    if (jc < jend && jc >= x.skip_n) {
      const double zr = zz[2 * jj], zi = zz[2 * jj + 1];
      double2* dst = x.Cz + x.crow + jc * x.ldc;
      if (p.mode == EPI_STORE) {
        if (p.ar == 1.0 && p.ai == 0.0) *dst = make_double2(zr, zi);
        else *dst = make_double2(p.ar * zr - p.ai * zi, p.ar * zi + p.ai * zr);
      } else if (p.mode == EPI_LU) {
        *dst = make_double2(cv[jj].x - zr, cv[jj].y - zi);
      } else if (p.mode == EPI_IMINUS) {
        *dst = make_double2((jc == x.grow ? 1.0 : 0.0) - zr, 0.0 - zi);
      } else {
        const double xr = p.ar * zr - p.ai * zi, xi = p.ar * zi + p.ai * zr;
        const double yr = p.br * cv[jj].x - p.bi * cv[jj].y, yi = p.br * cv[jj].y + p.bi * cv[jj].x;
        *dst = make_double2(xr + yr, xi + yi);
      }
    }
  }
  return true;
}

// Variant of epilogue_fast processing the 16 columns in two halves of 8: per half, the
// group accumulators stream through a double-buffered TMEM load (group g + 1 in flight while
// group g is folded) and the half's C values are loaded before its drain; the accumulators are
// released during the second half.
template <int G>
__device__ __forceinline__ bool epilogue_halves(const GemmParams& p, const EpiCtx& x, uint64_t* acc_empty, bool magic,
                                                int lane, ChunkWait& cw) {
  constexpr int NH = G < 4 ? G : 4;
  constexpr int NL = G - NH;
  constexpr int S8 = 8 * NL;
  constexpr int BN = 64;
  const bool needC = p.mode == EPI_LU || p.mode == EPI_GENERAL;
  const int jc0 = (x.n0 + x.c0) / 2;
  const int jend = min(min(jc0 + 8, (x.n2_z + 1) / 2), x.jlim);
  const bool active = x.rowok && max(jc0, x.skip_n) < jend;
  if (!__any_sync(0xffffffffu, active)) return release_unread<G>(acc_empty, cw, lane);
  if (!cw.next()) return false;                      // one exactness chunk (at most two K-blocks)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int jh = jc0 + 4 * half;                     // first complex column of this half
    double2 cv[4];
    int fe[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jc = jh + q;
      const bool w = active && jc < jend && jc >= x.skip_n;
      fe[q] = jc < jend ? p.f[x.z * p.f_stride + jc] : 0;
      cv[q] = (needC && w) ? x.Cz[x.crow + jc * x.ldc] : make_double2(0.0, 0.0);
    }
    long long H[8], L[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { H[j] = 0; L[j] = 0; }
    uint32_t va[8], vb[8];
    tmem_ld8(x.tbase + 8 * half, va);
    tmem_wait_ld();
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      uint32_t (&cur)[8] = (gi & 1) ? vb : va;
      uint32_t (&nxt)[8] = (gi & 1) ? va : vb;
      if (gi + 1 < G) tmem_ld8(x.tbase + (gi + 1) * BN + 8 * half, nxt);
      if (half == 1) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[gi]);     // both halves of group gi are read
      }
      const int w = gi < NH ? (1 << (8 * (NH - 1 - gi))) : (1 << (8 * (NL - 1 - (gi - NH))));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long a = static_cast<long long>(acc_to_int(cur[j], magic)) * w;
        if (gi < NH) H[j] += a; else L[j] += a;
      }
      if (gi + 1 < G) tmem_wait_ld();
    }
    if (active) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jc = jh + q;
        if (jc < jend && jc >= x.skip_n) {
          const int E = x.er + fe[q];
          double zz[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) zz[h] = round_hl_jam<S8>(H[2 * q + h], L[2 * q + h], E);
          double2* dst = x.Cz + x.crow + jc * x.ldc;
          if (p.mode == EPI_STORE) {
            if (p.ar == 1.0 && p.ai == 0.0) *dst = make_double2(zz[0], zz[1]);
            else *dst = make_double2(p.ar * zz[0] - p.ai * zz[1], p.ar * zz[1] + p.ai * zz[0]);
          } else if (p.mode == EPI_LU) {
            *dst = make_double2(cv[q].x - zz[0], cv[q].y - zz[1]);
          } else if (p.mode == EPI_IMINUS) {
            *dst = make_double2((jc == x.grow ? 1.0 : 0.0) - zz[0], 0.0 - zz[1]);
          } else {
            const double xr = p.ar * zz[0] - p.ai * zz[1], xi = p.ar * zz[1] + p.ai * zz[0];
            const double yr = p.br * cv[q].x - p.bi * cv[q].y, yi = p.br * cv[q].y + p.bi * cv[q].x;
            *dst = make_double2(xr + yr, xi + yi);
          }
        }
      }
    }
  }
  return true;
}

// RN-even of V 2^E for a two's-complement V with |V| < 2^63 (the exact sum when it fits in 64
// bits).  The int64 -> binary64 conversion is that rounding (RN-even of the integer to 53
// bits); while the result stays normal, the scaling by 2^E is exact and is an addition to the
// exponent field.  Results outside the normal range take the general routine, which rounds
// once at the subnormal position.
__device__ __forceinline__ double round_v64(long long V, int E) {
  const double d = __ll2double_rn(V);
  const long long bits = __double_as_longlong(d);
  const int ed = static_cast<int>((bits >> 52) & 0x7FF);
  if (ed == 0) return d;                                // V = 0
  if (ed + E < 1 || ed + E > 2046) return round_scaled_dev(static_cast<__int128>(V), E);
  return __longlong_as_double(bits + (static_cast<long long>(E) << 52));
}

// Epilogue of one 128 x 64 tile when the exact sum of every output fits in 64 bits: G <= 5
// groups, ceil(log2(terms)) + 14 + 8 (G - 1) + 1 <= 63 over all the tile's exactness chunks
// (checked on the host).  Chunk after chunk, every group is folded into one int64 per stacked
// column with the weight 2^(8 (G - 1 - g)) and its accumulator released; then the 16 sums are
// rounded and all of the thread's C values requested at once and combined.
template <int G>
__device__ __forceinline__ bool epilogue_fast64(const GemmParams& p, const EpiCtx& x, uint64_t* acc_empty,
                                                uint32_t magic_mask, int lane, ChunkWait& cw) {
  constexpr int BN = 64;
  const bool needC = p.mode == EPI_LU || p.mode == EPI_GENERAL;
  const int jc0 = (x.n0 + x.c0) / 2;                  // this thread's 8 complex columns
  const int jend = min(min(jc0 + 8, (x.n2_z + 1) / 2), x.jlim);
  const bool active = x.rowok && max(jc0, x.skip_n) < jend;
  if (!__any_sync(0xffffffffu, active)) return release_unread<G>(acc_empty, cw, lane);
  long long V[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) V[j] = 0;
  for (int c = 0; c < cw.nchunks; ++c) {
    if (!cw.next()) return false;
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      uint32_t v[8], u[8];
      tmem_ld8(x.tbase + gi * BN, v);
      tmem_ld8(x.tbase + gi * BN + 8, u);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[gi]);         // group gi may be overwritten now
      const long long w = 1ll << (8 * (G - 1 - gi));
      const bool mg = (magic_mask >> gi) & 1u;
      fold8(V, v, w, mg);
      fold8(V + 8, u, w, mg);
    }
  }
  if (!active) return true;
  // the 16 roundings (column exponents from memory; I - Z: RN(-V) = -RN(V), so the
  // off-diagonal outputs 0 - z need no binary64 operation), then every C value of the thread
  // requested at once, combined and written
  const bool negate = p.mode == EPI_IMINUS;
  double zz[16];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int jc = jc0 + jj;
    const int E = x.er + (jc < jend ? p.f[x.z * p.f_stride + jc] : 0);
    zz[2 * jj] = round_v64(negate ? -V[2 * jj] : V[2 * jj], E);
    zz[2 * jj + 1] = round_v64(negate ? -V[2 * jj + 1] : V[2 * jj + 1], E);
  }
  double2 cv[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int jc = jc0 + jj;
    cv[jj] = (needC && jc < jend && jc >= x.skip_n) ? x.Cz[x.crow + jc * x.ldc] : make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int jc = jc0 + jj;
    if (jc < jend && jc >= x.skip_n) {
      double2* dst = x.Cz + x.crow + jc * x.ldc;
      const double zr = zz[2 * jj], zi = zz[2 * jj + 1];
      if (p.mode == EPI_STORE) {
        if (p.ar == 1.0 && p.ai == 0.0) *dst = make_double2(zr, zi);
        else *dst = make_double2(p.ar * zr - p.ai * zi, p.ar * zi + p.ai * zr);
      } else if (p.mode == EPI_LU) {
        *dst = make_double2(cv[jj].x - zr, cv[jj].y - zi);
      } else if (p.mode == EPI_IMINUS) {
        *dst = make_double2(jc == x.grow ? 1.0 + zr : zr, zi);   // zr, zi hold -z
      } else {
        const double xr = p.ar * zr - p.ai * zi, xi = p.ar * zi + p.ai * zr;
        const double yr = p.br * cv[jj].x - p.bi * cv[jj].y, yi = p.br * cv[jj].y + p.bi * cv[jj].x;
        *dst = make_double2(xr + yr, xi + yi);
      }
    }
  }
  return true;
}

// SF = 0: the slice count, pair schedule and epilogue variant are chosen at run time.  SF > 0:
// an instance for S = SF with the triangular pair set only, whose MMA issuer and epilogue
// contain just that schedule and group count -- the tensor pipe is fed markedly faster from
// the compact code (about 67 instead of 100 cycles per 128 x 64 x 16 MMA in a probe of the
// same issue loop) and the epilogue warps run a fraction of the instructions' footprint.
template <int BN, int SF, bool KS>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ GemmParams p) {
  // Persistent: CTA b handles tiles b, b + gridDim.x, ... (column tile fastest, then row
  // tile, then problem).  All three roles walk the same tile sequence.
  constexpr int COLS = BN / 4;            // stacked columns per epilogue thread
  const bool single = p.m == nullptr;
  const int ntx = p.ntx, nty = p.nty;
  // KS instances run split K (p.ksplit units per tile); the others one unit per tile
  const int ks = KS ? (p.ksplit > 1 ? p.ksplit : 1) : 1;
  const int ntiles = (p.tile_prefix ? p.tile_prefix[p.batch] : p.tpp * p.batch) * ks;
  // work unit u: tile u / ks, exactness chunks [c0, c1) of its K
  auto unit_chunks = [&](int u, int nch, int& c0, int& c1) {
    const int sp = u - (u / ks) * ks;
    c0 = sp * nch / ks;
    c1 = (sp + 1) * nch / ks;
  };

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int S = SF > 0 ? SF : p.S;
  const int G = SF > 0 ? SF : p.ngroups;
  const uint32_t a_bytes = static_cast<uint32_t>(S) * GEMM_BM * 32;
  const uint32_t b_bytes = static_cast<uint32_t>(S) * BN * 32;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int nstage = p.nstage;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + nstage * stage_bytes);
  uint64_t* empty = full + nstage;
  uint64_t* acc_full = empty + nstage;
  uint64_t* acc_empty = acc_full + 1;          // one per group accumulator
  uint64_t* done_bar = acc_empty + 16;
  uint64_t* stall_bar = done_bar + 1;          // the test hook's barrier: no thread arrives at it
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(stall_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    mbar_init(acc_full, 1);
    for (int i = 0; i < 16; ++i) mbar_init(&acc_empty[i], GEMM_EPI_WARPS);
    mbar_init(done_bar, 1);
    mbar_init(stall_bar, 1);
    *abort_flag = 0;
    mbar_fence_init();
    prefetch_tensormap(&tmA);
    prefetch_tensormap(&tmB);
  }
  if (warp == 1) tmem_alloc(tmem_holder, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  if (p.stall_cycles > 0) {
    // failure-path test: one thread's bounded wait runs out (OZK_ERR_TIMEOUT, abort flag set)
    // before any TMA copy or MMA has been issued; every role then skips its loop
    if (threadIdx.x == 32) mbar_wait(stall_bar, 0, p.status, abort_flag, p.stall_cycles);
    __syncthreads();
  }
  const bool stalled = *abort_flag != 0;

  const int nkb = p.kblocks;
  const int nchunks = (nkb + p.chunk_kb - 1) / p.chunk_kb;

  // tile decode.  With exact enumeration (tile_prefix), problem z owns tiles [prefix[z],
  // prefix[z + 1]) laid out by box_tiles.  Otherwise problem z owns tiles [z tpp, (z + 1) tpp)
  // of the largest problem's grid: the tile rows below its skip box (all columns, column tile
  // fastest), then the tiles right of the box in the rows beside it; tiles wholly inside the
  // box are never enumerated.  Returns false for indices past the problem's own tiles or
  // outside its extent (skipped by all roles alike).
  auto tile_of = [&](int t, int& z, int& m0, int& n0, int& m_z, int& n2_z) -> bool {
    if (p.tile_prefix) {
      // exact enumeration: problem z owns tiles [prefix[z], prefix[z + 1]) of its own grid
      int lo = 0, hi = p.batch;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (p.tile_prefix[mid] <= t) lo = mid; else hi = mid;
      }
      z = lo;
      const int r = t - p.tile_prefix[z];
      m_z = p.m[z];
      n2_z = 2 * p.n[z];
      const BoxTiles bt = box_tiles(m_z, n2_z, p.skm ? p.skm[z] : 0, p.skn ? p.skn[z] : 0, BN);
      if (r < bt.ku * bt.xu) {                  // beside the box (rows clipped at its edge)
        const int y = r / bt.xu;
        m0 = y * GEMM_BM;
        n0 = bt.n0u + (r - y * bt.xu) * BN;
        m_z = bt.mu;
      } else {                                  // below the box, or the whole grid
        const int r2 = r - bt.ku * bt.xu, y = r2 / bt.ntx;
        m0 = bt.m0l + y * GEMM_BM;
        n0 = (r2 - y * bt.ntx) * BN;
      }
      return true;
    }
    z = t / p.tpp;
    const int r = t - z * p.tpp;
    m_z = single ? p.m1 : p.m[z];
    n2_z = 2 * (single ? p.n1 : p.n[z]);
    const int km = single ? p.skm1 : (p.skm ? p.skm[z] : 0);
    const int kn = single ? p.skn1 : (p.skn ? p.skn[z] : 0);
    const int ky = min(km / GEMM_BM, nty), kx = min((2 * kn) / BN, ntx);
    const int count1 = (nty - ky) * ntx;
    int x, y;
    if (r < count1) {
      y = ky + r / ntx;
      x = r - (y - ky) * ntx;
    } else {
      const int w = ntx - kx, r2 = r - count1;
      if (w <= 0 || r2 >= ky * w) return false;
      y = r2 / w;
      x = kx + (r2 - y * w);
    }
    m0 = y * GEMM_BM;
    n0 = x * BN;
    return m0 < m_z && n0 < n2_z;
  };

  // the 20 warps start with 96 registers each (61440 for the CTA); warpgroup 0 keeps 64 and the
  // epilogue warpgroups take 104 (128 x 64 + 512 x 104 = 61440)
  if (warp < GEMM_CTRL_WARPS) {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(GEMM_CTRL_REGS));
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: one ring of stages across all tiles
      uint32_t kbc = 0;
      bool ok = !stalled;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int z, m0, n0, m_z, n2_z;
        if (!tile_of(t / ks, z, m0, n0, m_z, n2_z)) continue;
        int za = z, ra = 0;
        if (p.remap) { const int2 rm = p.remap[z]; za = rm.x; ra = rm.y; }
        int c0, c1;
        unit_chunks(t, nchunks, c0, c1);
        const int kbe = min(nkb, c1 * p.chunk_kb);
        for (int kb = c0 * p.chunk_kb; kb < kbe; ++kb, ++kbc) {
          const int stage = kbc % nstage;
          const uint32_t ph = kbc / nstage;
          if (kbc >= static_cast<uint32_t>(nstage) && !mbar_wait(&empty[stage], (ph - 1) & 1, p.status, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * stage_bytes;
          mbar_arrive_expect_tx(&full[stage], stage_bytes);
          tma_load_3d(&tmA, sa, &full[stage], kb * 16, ra + m0, za * S);
          tma_load_3d(&tmB, sa + a_bytes, &full[stage], kb * 16, n0, za * S);
        }
      }
      if (!ok || *abort_flag) {
        // another role gave up: let the copies this thread issued land before the CTA exits
        for (uint32_t k = kbc > static_cast<uint32_t>(nstage) ? kbc - nstage : 0u; k < kbc; ++k) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[k % nstage], (k / nstage) & 1) && clock64() - t0 < kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer.  Group g's accumulator of chunk cc may be overwritten
      // once the epilogue released it for chunk cc - 1 (per-group barrier), so the MMAs of
      // the next tile overlap the reconstruction of the current one.
      const uint32_t idesc = idesc_f16_f32(GEMM_BM, BN);
      uint32_t kbc = 0, cc = 0;
      bool ok = !stalled;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int z, m0, n0, m_z, n2_z;
        if (!tile_of(t / ks, z, m0, n0, m_z, n2_z)) continue;
        int cb, ce;
        unit_chunks(t, nchunks, cb, ce);
        for (int c = cb; c < ce && ok; ++c, ++cc) {
          const int kb0 = c * p.chunk_kb;
          const int kb1 = min(nkb, kb0 + p.chunk_kb);
          for (int kb = kb0; kb < kb1 && ok; ++kb, ++kbc) {
            const int stage = kbc % nstage;
            if (!mbar_wait(&full[stage], (kbc / nstage) & 1, p.status, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + stage * stage_bytes);
            const uint32_t sb = sa + a_bytes;
            const uint64_t da = smem_desc_sw32(sa), db = smem_desc_sw32(sb);
            if constexpr (SF > 0)
              ok = issue_kblock_any<SF, false, BN>(kb == kb0, tmem, static_cast<uint32_t>(da), static_cast<uint32_t>(db),
                                                   static_cast<uint32_t>(da >> 32), idesc, acc_empty, (cc - 1) & 1,
                                                   cc > 0, p.status, abort_flag);
            else if (dispatch_covers<BN>(p, S))
              ok = issue_dispatch<BN>(S, p.fullset != 0, kb == kb0, tmem, static_cast<uint32_t>(da),
                                      static_cast<uint32_t>(db), static_cast<uint32_t>(da >> 32), idesc, acc_empty,
                                      (cc - 1) & 1, cc > 0, p.status, abort_flag);
            else
              ok = issue_runtime<BN>(p, kb == kb0, tmem, static_cast<uint32_t>(da), static_cast<uint32_t>(db),
                                     static_cast<uint32_t>(da >> 32), idesc, acc_empty, (cc - 1) & 1, cc > 0,
                                     abort_flag);
            if (!ok) break;
            mma_commit(&empty[stage]);
          }
          if (ok) mma_commit(acc_full);
        }
      }
      // make sure no MMA is still in flight before TMEM is released
      mma_commit(done_bar);
      const long long t0 = clock64();
      while (!mbar_try_wait(done_bar, 0)) {
        if (clock64() - t0 > kWaitBudget) { flag_error(p.status, OZK_ERR_TIMEOUT); break; }
      }
    }
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(GEMM_EPI_REGS));
    // ---------------- epilogue: 16 warps = 4 TMEM lane quadrants x 4 column slabs
    const int quad = warp & 3;
    const int slab = (warp - GEMM_CTRL_WARPS) >> 2;
    const int c0 = slab * COLS;                  // first local stacked column of this thread
    const uint32_t tbase = tmem + (static_cast<uint32_t>(quad * 32) << 16) + c0;
    const bool magic = p.magic != 0;
    const uint32_t magic_mask = magic ? 0xFFFFFFFFu : static_cast<uint32_t>(p.magic_mask);
    const bool horner = nchunks == 1;
    uint32_t cc = 0;
    bool ok = !stalled;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int z, m0, n0, m_z, n2_z;
      if (!tile_of(t / ks, z, m0, n0, m_z, n2_z)) continue;
      int ucb, uce;
      unit_chunks(t, nchunks, ucb, uce);
      const int unch = uce - ucb;                // exactness chunks of this unit
      int za = z, ra = 0;
      if (p.remap) { const int2 rm = p.remap[z]; za = rm.x; ra = rm.y; }
      const int row = m0 + quad * 32 + lane;
      const bool rowok = row < m_z;
      if constexpr (COLS == 16) {
        if (G <= 8 && p.mode != EPI_GROUPS && p.mode != EPI_RESIDUES) {
          EpiCtx x;
          x.row = row; x.z = za; x.m_z = m_z; x.n2_z = n2_z; x.n0 = n0; x.c0 = c0; x.tbase = tbase;
          x.rowok = rowok;
          x.skip_n = (row < (single ? p.skm1 : (p.skm ? p.skm[z] : 0))) ? (single ? p.skn1 : p.skn[z]) : 0;
          out_row(p, single, z, row, za, ra, x.rowok, x.Cz, x.crow, x.grow, x.ldc, x.jlim);
          x.er = x.rowok ? p.e[za * p.e_stride + ra + row] + p.base_exp : 0;
          x.sp = t - (t / ks) * ks;
          ChunkWait cw{acc_full, unch, &cc, p.status, abort_flag};
          // short K (at most two K-blocks per tile): the epilogue bounds the tile, and the
          // two-halves variant with streamed TMEM loads is faster (1.18x on 1024 x 1040 x 16
          // tiles); longer K: the group-wise drain that releases accumulators earliest (1.14x
          // on 976 x 976 x 64)
          const bool halves = p.kblocks <= 2 && nchunks == 1;
          bool e_ok;
          if constexpr (SF > 0) {
            if (SF <= 5 && p.fit64) e_ok = epilogue_fast64<(SF <= 5 ? SF : 5)>(p, x, acc_empty, magic_mask, lane, cw);
            else if (halves) e_ok = epilogue_halves<SF>(p, x, acc_empty, magic, lane, cw);
            else e_ok = epilogue_fast<SF, KS>(p, x, acc_empty, magic, lane, cw);
          } else if (p.fit64 && G <= 5) {
            switch (G) {
              case 1: e_ok = epilogue_fast64<1>(p, x, acc_empty, magic_mask, lane, cw); break;
              case 2: e_ok = epilogue_fast64<2>(p, x, acc_empty, magic_mask, lane, cw); break;
              case 3: e_ok = epilogue_fast64<3>(p, x, acc_empty, magic_mask, lane, cw); break;
              case 4: e_ok = epilogue_fast64<4>(p, x, acc_empty, magic_mask, lane, cw); break;
              default: e_ok = epilogue_fast64<5>(p, x, acc_empty, magic_mask, lane, cw); break;
            }
          } else if (halves) {
            switch (G) {
              case 1: e_ok = epilogue_halves<1>(p, x, acc_empty, magic, lane, cw); break;
              case 2: e_ok = epilogue_halves<2>(p, x, acc_empty, magic, lane, cw); break;
              case 3: e_ok = epilogue_halves<3>(p, x, acc_empty, magic, lane, cw); break;
              case 4: e_ok = epilogue_halves<4>(p, x, acc_empty, magic, lane, cw); break;
              case 5: e_ok = epilogue_halves<5>(p, x, acc_empty, magic, lane, cw); break;
              case 6: e_ok = epilogue_halves<6>(p, x, acc_empty, magic, lane, cw); break;
              case 7: e_ok = epilogue_halves<7>(p, x, acc_empty, magic, lane, cw); break;
              default: e_ok = epilogue_halves<8>(p, x, acc_empty, magic, lane, cw); break;
            }
          } else {
            switch (G) {
              case 1: e_ok = epilogue_fast<1, KS>(p, x, acc_empty, magic, lane, cw); break;
              case 2: e_ok = epilogue_fast<2, KS>(p, x, acc_empty, magic, lane, cw); break;
              case 3: e_ok = epilogue_fast<3, KS>(p, x, acc_empty, magic, lane, cw); break;
              case 4: e_ok = epilogue_fast<4, KS>(p, x, acc_empty, magic, lane, cw); break;
              case 5: e_ok = epilogue_fast<5, KS>(p, x, acc_empty, magic, lane, cw); break;
              case 6: e_ok = epilogue_fast<6, KS>(p, x, acc_empty, magic, lane, cw); break;
              case 7: e_ok = epilogue_fast<7, KS>(p, x, acc_empty, magic, lane, cw); break;
              default: e_ok = epilogue_fast<8, KS>(p, x, acc_empty, magic, lane, cw); break;
            }
          }
          if (!e_ok) { ok = false; break; }
          continue;
        }
      }
      if constexpr (SF > 0) continue;            // compile-time instances take only the fast epilogues
      __int128 T[COLS];
#pragma unroll
      for (int j = 0; j < COLS; ++j) T[j] = 0;
      for (int c = 0; c < nchunks; ++c, ++cc) {
        if (!mbar_wait(acc_full, cc & 1, p.status, abort_flag)) { ok = false; break; }
        tc_fence_after();
        for (int gi = 0; gi < G; ++gi) {
          uint32_t v[COLS];
          if constexpr (COLS == 16) tmem_ld16(tbase + gi * BN, v); else tmem_ld8(tbase + gi * BN, v);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[gi]);       // group gi may be overwritten now
          if (p.mode == EPI_RESIDUES) {
            // this chunk's exact integer value of group gi (|v| <= 2^24), added to the product
            if (rowok) {
              int* dst = p.resid + ((static_cast<long long>(z) * G + gi) * m_z + row) * p.ldres;
#pragma unroll
              for (int j = 0; j < COLS; ++j) {
                const int col = n0 + c0 + j;
                if (col < n2_z) atomicAdd(&dst[col], __float2int_rn(__uint_as_float(v[j])));
              }
            }
          } else if (p.mode == EPI_GROUPS) {
            if (z == 0 && rowok) {
#pragma unroll
              for (int j = 0; j < COLS; ++j) {
                const int col = n0 + c0 + j;
                if (col < n2_z) {
                  const long long iv = __float2int_rn(__uint_as_float(v[j]));
                  atomicAdd(reinterpret_cast<unsigned long long*>(&p.groups[(static_cast<long long>(gi) * m_z + row) * n2_z + col]),
                            static_cast<unsigned long long>(iv));
                }
              }
            }
          } else if (horner) {
            // one chunk: Horner over the groups, highest weight first, 8-bit steps
#pragma unroll
            for (int j = 0; j < COLS; ++j) T[j] = (T[j] << 8) + static_cast<__int128>(acc_to_int(v[j], magic));
          } else {
            const int w = 8 * (G - 1 - gi);
#pragma unroll
            for (int j = 0; j < COLS; ++j) T[j] += static_cast<__int128>(__float2int_rn(__uint_as_float(v[j]))) << w;
          }
        }
      }
      if (!ok) break;
      double2* Cz = nullptr;
      long long crow = 0, ldc = 0;
      int grow = 0, jlim = 0;
      bool rowok2 = rowok;
      if (p.mode != EPI_GROUPS && p.mode != EPI_RESIDUES)
        out_row(p, single, z, row, za, ra, rowok2, Cz, crow, grow, ldc, jlim);
      if (p.mode != EPI_GROUPS && p.mode != EPI_RESIDUES && rowok2) {
        const int er = p.e[za * p.e_stride + ra + row] + p.base_exp;
        const int skip_n = (row < (single ? p.skm1 : (p.skm ? p.skm[z] : 0))) ? (single ? p.skn1 : p.skn[z]) : 0;
#pragma unroll
        for (int j = 0; j < COLS; j += 2) {
          const int jc = (n0 + c0 + j) >> 1;          // complex column
          if (2 * jc < n2_z && jc >= skip_n && jc < jlim) {
            const int E = er + p.f[za * p.f_stride + jc];
            const double zr = round_scaled_dev(T[j], E);
            const double zi = round_scaled_dev(T[j + 1], E);
            double2* dst = Cz + crow + jc * ldc;
            if (p.mode == EPI_STORE) {
              if (p.ar == 1.0 && p.ai == 0.0) *dst = make_double2(zr, zi);
              else *dst = make_double2(p.ar * zr - p.ai * zi, p.ar * zi + p.ai * zr);
            } else if (p.mode == EPI_IMINUS) {
              *dst = make_double2((jc == grow ? 1.0 : 0.0) - zr, 0.0 - zi);
            } else if (p.mode == EPI_LU) {
              const double2 cv = *dst;
              *dst = make_double2(cv.x - zr, cv.y - zi);
            } else {
              const double2 cv = *dst;
              const double xr = p.ar * zr - p.ai * zi, xi = p.ar * zi + p.ai * zr;
              const double yr = p.br * cv.x - p.bi * cv.y, yi = p.br * cv.y + p.bi * cv.x;
              *dst = make_double2(xr + yr, xi + yi);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

size_t gemm_smem_bytes(int S, int BN, int nstage) {
  const size_t stage = static_cast<size_t>(S) * (GEMM_BM + BN) * 32;
  return 1024 + nstage * stage + (2 * nstage + 19) * 8 + 16;
}

static int num_sms() {
  static const int n = [] {                       // initialised once, thread-safe
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
  }();
  return n;
}

int gpu_sm_count() { return num_sms(); }

void launch_slice_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmParams& p0, int BN,
                       int max_m, int max_n, int batch, cudaStream_t st) {
  GemmParams p = p0;
  p.ntx = (2 * max_n + BN - 1) / BN;
  p.nty = (max_m + GEMM_BM - 1) / GEMM_BM;
  p.batch = batch;
  const int ky = std::min(p.box_m / GEMM_BM, p.nty), kx = std::min((2 * p.box_n) / BN, p.ntx);
  p.tpp = p.ntx * p.nty - kx * ky;
  // with exact enumeration the tile count is on the device: one persistent CTA per SM
  const long long ntiles = static_cast<long long>(p.tpp) * batch * std::max(1, p.ksplit);
  const int grid = static_cast<int>(std::min<long long>(ntiles, num_sms()));
  const size_t smem = gemm_smem_bytes(p.S, BN, p.nstage);
  // the compile-time instances hold only the fast epilogues (no integer group dumps)
  const bool tri = BN == 64 && !p.fullset && !p.diag_pairs && p.mode != EPI_GROUPS && p.mode != EPI_RESIDUES;
  const bool ks = p.ksplit > 1;                 // split K: its own instances (the unit bookkeeping
                                                // costs the others registers)
#define OZK_LAUNCH(BN_, SF_, KS_)                                                                          \
  do {                                                                                                     \
    cudaFuncSetAttribute(slice_gemm_kernel<BN_, SF_, KS_>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                         static_cast<int>(smem));                                                          \
    slice_gemm_kernel<BN_, SF_, KS_><<<grid, GEMM_THREADS, smem, st>>>(ta, tb, p);                         \
  } while (0)
  if (tri && p.S == 5 && !ks) {
    // the slice count the selector picks for most KKR GEMMs: a compact instance
    OZK_LAUNCH(64, 5, false);
  } else if (tri && p.S == 7) {
    // 55 bits, the precision of the batched contour workload
    if (ks) OZK_LAUNCH(64, 7, true);
    else OZK_LAUNCH(64, 7, false);
  } else if (BN == 64) {
    if (ks) OZK_LAUNCH(64, 0, true);
    else OZK_LAUNCH(64, 0, false);
  } else {
    OZK_LAUNCH(32, 0, false);
  }
#undef OZK_LAUNCH
  record_launch();
}

// Split K of a single problem: output (row, complex column jc) is the sum over the units of
// their exact 64-bit halves (H, L) of the real and imaginary stacked columns 2 jc, 2 jc + 1 (the
// integer sums are split between the units, so their sum is the sum the one-unit epilogue
// forms), rounded once by the same routine and combined with C in the slice GEMM's modes.
template <int G>
__global__ void __launch_bounds__(256) finish_split_kernel(const __grid_constant__ GemmParams p) {
  constexpr int NH = G < 4 ? G : 4;
  constexpr int NL = G - NH;
  constexpr int S8 = 8 * NL;
  const int m = p.m1, n = p.n1, n2 = 2 * n;
  const long long total = static_cast<long long>(m) * n;
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int row = static_cast<int>(idx % m), jc = static_cast<int>(idx / m);
    long long Hr = 0, Lr = 0, Hi = 0, Li = 0;
    for (int sp = 0; sp < p.ksplit; ++sp) {
      const longlong2 a = p.part[(static_cast<long long>(sp) * n2 + 2 * jc) * m + row];
      const longlong2 b = p.part[(static_cast<long long>(sp) * n2 + 2 * jc + 1) * m + row];
      Hr += a.x; Lr += a.y; Hi += b.x; Li += b.y;
    }
    const int E = p.e[row] + p.base_exp + p.f[jc];
    const double zr = round_hl_jam<S8>(Hr, Lr, E), zi = round_hl_jam<S8>(Hi, Li, E);
    double2* dst = p.C1 + row + static_cast<long long>(jc) * p.ldc1;
    if (p.mode == EPI_STORE) {
      if (p.ar == 1.0 && p.ai == 0.0) *dst = make_double2(zr, zi);
      else *dst = make_double2(p.ar * zr - p.ai * zi, p.ar * zi + p.ai * zr);
    } else if (p.mode == EPI_LU) {
      const double2 cv = *dst;
      *dst = make_double2(cv.x - zr, cv.y - zi);
    } else {
      const double2 cv = *dst;
      const double xr = p.ar * zr - p.ai * zi, xi = p.ar * zi + p.ai * zr;
      const double yr = p.br * cv.x - p.bi * cv.y, yi = p.br * cv.y + p.bi * cv.x;
      *dst = make_double2(xr + yr, xi + yi);
    }
  }
}

void launch_finish_split(const GemmParams& p, cudaStream_t st) {
  const long long total = static_cast<long long>(p.m1) * p.n1;
  const unsigned blocks = static_cast<unsigned>(std::min<long long>((total + 255) / 256, 8L * num_sms()));
  switch (p.ngroups) {
    case 1: finish_split_kernel<1><<<blocks, 256, 0, st>>>(p); break;
    case 2: finish_split_kernel<2><<<blocks, 256, 0, st>>>(p); break;
    case 3: finish_split_kernel<3><<<blocks, 256, 0, st>>>(p); break;
    case 4: finish_split_kernel<4><<<blocks, 256, 0, st>>>(p); break;
    case 5: finish_split_kernel<5><<<blocks, 256, 0, st>>>(p); break;
    case 6: finish_split_kernel<6><<<blocks, 256, 0, st>>>(p); break;
    case 7: finish_split_kernel<7><<<blocks, 256, 0, st>>>(p); break;
    default: finish_split_kernel<8><<<blocks, 256, 0, st>>>(p); break;
  }
  record_launch();
}

// Tile counts of the problems of a batched GEMM (each over its own grid, tiles wholly inside
// its skip box left out) and their exclusive prefix sums: one CTA, chunks of 1024 problems.
__global__ void __launch_bounds__(1024) tile_prefix_kernel(const int* __restrict__ m, const int* __restrict__ n,
                                                           const int* __restrict__ skm, const int* __restrict__ skn,
                                                           int batch, int BN, int* __restrict__ out) {
  __shared__ int part[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < batch; base += 1024) {
    const int z = base + static_cast<int>(threadIdx.x);
    int c = 0;
    if (z < batch && m[z] > 0 && n[z] > 0) {
      const BoxTiles bt = box_tiles(m[z], 2 * n[z], skm ? skm[z] : 0, skn ? skn[z] : 0, BN);
      c = bt.ku * bt.xu + bt.nl * bt.ntx;
    }
    part[threadIdx.x] = c;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {          // inclusive scan (Hillis-Steele)
      const int v = threadIdx.x >= static_cast<unsigned>(off) ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (z < batch) out[z] = carry + part[threadIdx.x] - c;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[batch] = carry;
}

void launch_tile_prefix(const GemmParams& p, int BN, int batch, int* out, cudaStream_t st) {
  tile_prefix_kernel<<<1, 1024, 0, st>>>(p.m, p.n, p.skm, p.skn, batch, BN, out);
  record_launch();
}

}  // namespace ozk
