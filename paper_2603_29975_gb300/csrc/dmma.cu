// Plain binary64 complex GEMM on the FP64 tensor path (mma.sync.m8n8k4.f64, "DMMA"): the
// native-precision baseline the emulation is compared against on the same GPU (the paper
// uses native FP64 GEMM as its ground truth, Sec. 3.2 and Sec. 4).
//
// C = alpha op(A) op(B) + beta C, column major.  A CTA computes a 32 x 32 complex tile with
// four warps (2 x 2), each warp a 16 x 16 tile of 2 x 2 blocks of 8 x 8.  Complex products
// are four real MMAs per block: Cr += Ar Br, Cr += (-Ai) Bi, Ci += Ar Bi, Ci += Ai Br.
#include <algorithm>

#include "ozk_params.cuh"

namespace ozk {

constexpr int DM_TILE = 32;
constexpr int DM_KT = 8;
constexpr int DM_THREADS = 128;



__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(DM_THREADS)
zgemm_dmma_kernel(const DmmaParams p) {
  __shared__ double Ar[DM_KT][DM_TILE + 1], Ai[DM_KT][DM_TILE + 1];
  __shared__ double Br[DM_KT][DM_TILE + 1], Bi[DM_KT][DM_TILE + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.y * DM_TILE, j0 = blockIdx.x * DM_TILE;
  const bool batched = p.tm != nullptr;
  const int z = blockIdx.z;
  const int m = batched ? p.tm[z] : p.m, n = batched ? p.tn[z] : p.n, kdim = batched ? p.tk[z] : p.k;
  if (i0 >= m || j0 >= n) return;                 // whole CTA outside this problem
  const double2* A = batched ? p.tA[z] : p.A;
  const double2* B = batched ? p.tB[z] : p.B;
  double2* C = batched ? p.tC[z] : p.C;
  const long long lda = batched ? p.tlda[z] : p.lda, ldb = batched ? p.tldb[z] : p.ldb;
  const long long ldc = batched ? p.tldc[z] : p.ldc;
  const int wr = (warp >> 1) * 16, wc = (warp & 1) * 16;
  const int g = lane >> 2, q = lane & 3;
  double cr[2][2][2] = {}, ci[2][2][2] = {};

  for (int l0 = 0; l0 < kdim; l0 += DM_KT) {
    // A tile: 32 rows x 8 k ; B tile: 8 k x 32 cols  (256 complex each, 2 per thread)
    for (int idx = tid; idx < DM_TILE * DM_KT; idx += DM_THREADS) {
      int r, l;
      if (!p.transa) { r = idx % DM_TILE; l = idx / DM_TILE; } else { l = idx % DM_KT; r = idx / DM_KT; }
      const int gi = i0 + r, gl = l0 + l;
      double2 v = make_double2(0.0, 0.0);
      if (gi < m && gl < kdim) v = p.transa ? A[gl + gi * lda] : A[gi + gl * lda];
      if (p.conja) v.y = -v.y;
      Ar[l][r] = v.x; Ai[l][r] = v.y;
    }
    for (int idx = tid; idx < DM_TILE * DM_KT; idx += DM_THREADS) {
      int c, l;
      if (!p.transb) { l = idx % DM_KT; c = idx / DM_KT; } else { c = idx % DM_TILE; l = idx / DM_TILE; }
      const int gj = j0 + c, gl = l0 + l;
      double2 v = make_double2(0.0, 0.0);
      if (gj < n && gl < kdim) v = p.transb ? B[gj + gl * ldb] : B[gl + gj * ldb];
      if (p.conjb) v.y = -v.y;
      Br[l][c] = v.x; Bi[l][c] = v.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DM_KT; kk += 4) {
      double far[2], fai[2], fan[2], fbr[2], fbi[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        far[a] = Ar[kk + q][wr + a * 8 + g];
        fai[a] = Ai[kk + q][wr + a * 8 + g];
        fan[a] = -fai[a];
      }
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        fbr[b] = Br[kk + q][wc + b * 8 + g];
        fbi[b] = Bi[kk + q][wc + b * 8 + g];
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          dmma(cr[a][b][0], cr[a][b][1], far[a], fbr[b]);
          dmma(cr[a][b][0], cr[a][b][1], fan[a], fbi[b]);
          dmma(ci[a][b][0], ci[a][b][1], far[a], fbi[b]);
          dmma(ci[a][b][0], ci[a][b][1], fai[a], fbr[b]);
        }
    }
    __syncthreads();
  }
  // epilogue: thread holds rows wr + a*8 + g, cols wc + b*8 + 2q + {0,1}
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gi = i0 + wr + a * 8 + g;
        const int gj = j0 + wc + b * 8 + 2 * q + h;
        if (gi < m && gj < n) {
          const double zr = cr[a][b][h], zi = ci[a][b][h];
          double2* dst = C + gi + gj * ldc;
          double xr = p.ar * zr - p.ai * zi, xi = p.ar * zi + p.ai * zr;
          if (p.br != 0.0 || p.bi != 0.0) {
            const double2 cv = *dst;
            xr += p.br * cv.x - p.bi * cv.y;
            xi += p.br * cv.y + p.bi * cv.x;
          }
          *dst = make_double2(xr, xi);
        }
      }
}

void launch_dmma(const DmmaParams& p, cudaStream_t st) {
  if (p.m <= 0 || p.n <= 0) return;
  dim3 grid((p.n + DM_TILE - 1) / DM_TILE, (p.m + DM_TILE - 1) / DM_TILE, p.tm ? std::max(p.batch, 1) : 1);
  zgemm_dmma_kernel<<<grid, DM_THREADS, 0, st>>>(p);
  record_launch();
}

__global__ void strided_ptrs_kernel(double2** out, int* ld, double2* base, long long stride, int ldv, int n) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n) {
    out[z] = base + z * stride;
    ld[z] = ldv;
  }
}

void launch_strided_ptrs(double2** out, int* ld, double2* base, long long stride, int ldv, int n, cudaStream_t st) {
  if (n <= 0) return;
  strided_ptrs_kernel<<<(n + 127) / 128, 128, 0, st>>>(out, ld, base, stride, ldv, n);
  record_launch();
}

}  // namespace ozk
