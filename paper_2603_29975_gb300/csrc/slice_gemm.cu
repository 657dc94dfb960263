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
//     accumulator per group (G groups x BN columns of the 512);
//   * warps 2..17 drain the accumulators.  Every product of two digits is an integer of
//     magnitude <= 2^14 and each accumulator receives at most 1024 of them per "exactness
//     chunk" of K, so every FP32 value is an exact integer <= 2^24.  The epilogue converts
//     it to int32 and adds it, shifted by its group weight 8 (g_max - g) bits, into a 128-bit
//     integer per output element; after the last chunk that integer times 2^(e_i + f_j + c)
//     is rounded once to binary64 with integer instructions only, then stored (C = Z), or
//     subtracted from C (LU update), or combined with alpha/beta.
// No FP64 instruction touches the products; the only binary64 arithmetic is the final
// subtraction / alpha-beta combination per element.
#include "ozk_params.cuh"

namespace ozk {

constexpr int GEMM_BM = 128;
constexpr int GEMM_EPI_WARPS = 16;
constexpr int GEMM_THREADS = (2 + GEMM_EPI_WARPS) * 32;


// RN-even of T * 2^E as binary64, integer instructions only (subnormals and overflow handled).
__device__ __forceinline__ double round_scaled_dev(__int128 T, int E) {
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const unsigned __int128 u = neg ? static_cast<unsigned __int128>(-T) : static_cast<unsigned __int128>(T);
  const unsigned long long hi = static_cast<unsigned long long>(u >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(u);
  // normalise to a 64-bit significand M (top bit set) with a sticky bit for the rest
  unsigned long long M;
  int nb;              // bit length of u
  bool sticky;
  if (hi) {
    const int lz = __clzll(hi);
    nb = 128 - lz;
    M = lz ? ((hi << lz) | (lo >> (64 - lz))) : hi;
    sticky = lz ? ((lo << lz) != 0ull) : (lo != 0ull);
  } else {
    const int lz = __clzll(lo);
    nb = 64 - lz;
    M = lo << lz;
    sticky = false;
  }
  // value = (M + sticky*) * 2^(E + nb - 64); ulp exponent of the result:
  const int Ep = E + nb - 64;
  int q = Ep + 11;                 // 64 - 53
  if (q < -1074) q = -1074;
  const int drop = q - Ep;         // >= 11
  unsigned long long keep, rem, half;
  if (drop < 64) {
    keep = M >> drop;
    rem = M & ((1ull << drop) - 1ull);
    half = 1ull << (drop - 1);
  } else if (drop == 64) {
    keep = 0ull; rem = M; half = 1ull << 63;
  } else {
    keep = 0ull; rem = 0ull; half = 1ull; sticky = sticky || (M != 0ull);  // far below half an ulp
  }
  const bool up = (rem > half) || (rem == half && (sticky || (keep & 1ull)));
  keep += up ? 1ull : 0ull;
  if (keep == 0ull) return neg ? -0.0 : 0.0;
  // keep <= 2^53; value = keep * 2^q; bits = ((q + 1074) << 52) + keep covers normals and
  // subnormals alike (a carry out of the significand bumps the exponent field)
  unsigned long long bits;
  if (q + 1074 >= 2047) {
    bits = 0x7FF0000000000000ull;   // overflow to infinity
  } else {
    bits = (static_cast<unsigned long long>(q + 1074) << 52) + keep;
    if (bits >= 0x7FF0000000000000ull) bits = 0x7FF0000000000000ull;
  }
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double(static_cast<long long>(bits));
}

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ GemmParams p) {
  constexpr int COLS = BN / 4;            // stacked columns per epilogue thread
  const int z = blockIdx.z;
  const bool single = p.m == nullptr;
  const int m_z = single ? p.m1 : p.m[z];
  const int n2_z = 2 * (single ? p.n1 : p.n[z]);
  const int m0 = blockIdx.y * GEMM_BM;
  const int n0 = blockIdx.x * BN;
  if (m0 >= m_z || n0 >= n2_z) return;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int S = p.S;
  const uint32_t a_bytes = static_cast<uint32_t>(S) * GEMM_BM * 32;
  const uint32_t b_bytes = static_cast<uint32_t>(S) * BN * 32;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int nstage = p.nstage;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + nstage * stage_bytes);
  uint64_t* empty = full + nstage;
  uint64_t* acc_full = empty + nstage;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done_bar = acc_empty + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, GEMM_EPI_WARPS);
    mbar_init(done_bar, 1);
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

  const int nkb = p.kblocks;
  const int nchunks = (nkb + p.chunk_kb - 1) / p.chunk_kb;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int stage = kb % nstage;
        const uint32_t round = kb / nstage;
        if (kb >= nstage && !mbar_wait(&empty[stage], (round - 1) & 1, p.status, abort_flag)) break;
        uint8_t* sa = smem + stage * stage_bytes;
        mbar_arrive_expect_tx(&full[stage], stage_bytes);
        tma_load_3d(&tmA, sa, &full[stage], kb * 16, m0, z * S);
        tma_load_3d(&tmB, sa + a_bytes, &full[stage], kb * 16, n0, z * S);
        issued = kb + 1;
      }
      if (*abort_flag) {
        // another role gave up: let the copies this thread issued land before the CTA exits
        for (int kb = max(0, issued - nstage); kb < issued; ++kb) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[kb % nstage], (kb / nstage) & 1) && clock64() - t0 < kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t idesc = idesc_f16_f32(GEMM_BM, BN);
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        if (c > 0) { ok = mbar_wait(acc_empty, (c - 1) & 1, p.status, abort_flag); if (!ok) break; }
        tc_fence_after();
        const int kb0 = c * p.chunk_kb;
        const int kb1 = min(nkb, kb0 + p.chunk_kb);
        for (int kb = kb0; kb < kb1; ++kb) {
          const int stage = kb % nstage;
          const uint32_t round = kb / nstage;
          if (!mbar_wait(&full[stage], round & 1, p.status, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * stage_bytes);
          const uint32_t sb = sa + a_bytes;
          for (int pi = 0; pi < p.npairs; ++pi) {
            const uint32_t s = p.ps[pi], t = p.pt[pi], g = p.pg[pi];
            const uint64_t ad = smem_desc_sw32(sa + s * (GEMM_BM * 32));
            const uint64_t bd = smem_desc_sw32(sb + t * (BN * 32));
            const uint32_t acc = (kb == kb0 && p.pfirst[pi]) ? 0u : 1u;
            mma_f16(tmem + g * BN, ad, bd, idesc, acc);
          }
          mma_commit(&empty[stage]);
        }
        if (ok) mma_commit(acc_full);
      }
      // make sure no MMA is still in flight before TMEM is released
      mma_commit(done_bar);
      const long long t0 = clock64();
      while (!mbar_try_wait(done_bar, 0)) {
        if (clock64() - t0 > kWaitBudget) { flag_error(p.status, OZK_ERR_TIMEOUT); break; }
      }
    }
  } else {
    // ---------------- epilogue: 16 warps = 4 TMEM lane quadrants x 4 column slabs
    const int quad = warp & 3;
    const int slab = (warp - 2) >> 2;
    const int row = m0 + quad * 32 + lane;
    const int c0 = slab * COLS;                  // first local stacked column of this thread
    const int G = p.ngroups;
    __int128 T[COLS];
#pragma unroll
    for (int j = 0; j < COLS; ++j) T[j] = 0;
    const uint32_t tbase = tmem + (static_cast<uint32_t>(quad * 32) << 16) + c0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(acc_full, c & 1, p.status, abort_flag)) { ok = false; break; }
      tc_fence_after();
      for (int gi = 0; gi < G; ++gi) {
        uint32_t v[COLS];
        if constexpr (COLS == 16) tmem_ld16(tbase + gi * BN, v); else tmem_ld8(tbase + gi * BN, v);
        tmem_wait_ld();
        if (p.mode == EPI_GROUPS) {
          if (z == 0 && row < m_z) {
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
        } else {
          const int w = 8 * (G - 1 - gi);
#pragma unroll
          for (int j = 0; j < COLS; ++j) {
            const int iv = __float2int_rn(__uint_as_float(v[j]));
            T[j] += static_cast<__int128>(iv) << w;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    if (ok && p.mode != EPI_GROUPS && row < m_z) {
      const int er = p.e[z * p.e_stride + row] + p.base_exp;
      double2* Cz = single ? p.C1 : p.C[z];
      const long long ldc = single ? p.ldc1 : p.ldc[z];
#pragma unroll
      for (int j = 0; j < COLS; j += 2) {
        const int jc = (n0 + c0 + j) >> 1;          // complex column
        if (2 * jc < n2_z) {
          const int E = er + p.f[z * p.f_stride + jc];
          const double zr = round_scaled_dev(T[j], E);
          const double zi = round_scaled_dev(T[j + 1], E);
          double2* dst = Cz + row + jc * ldc;
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
  return 1024 + nstage * stage + (2 * nstage + 3) * 8 + 16;
}

void launch_slice_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmParams& p, int BN,
                       int max_m, int max_n, int batch, cudaStream_t st) {
  const size_t smem = gemm_smem_bytes(p.S, BN, p.nstage);
  dim3 grid((2 * max_n + BN - 1) / BN, (max_m + GEMM_BM - 1) / GEMM_BM, batch);
  if (BN == 64) {
    cudaFuncSetAttribute(slice_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    slice_gemm_kernel<64><<<grid, GEMM_THREADS, smem, st>>>(ta, tb, p);
  } else {
    cudaFuncSetAttribute(slice_gemm_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    slice_gemm_kernel<32><<<grid, GEMM_THREADS, smem, st>>>(ta, tb, p);
  }
  record_launch();
}

}  // namespace ozk
