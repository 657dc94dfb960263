// KKR kernels around the emulated GEMMs (paper Sec. 3.2: LU-based inversion of the
// multiple scattering matrix M = I - t G, whose central block gives tau_00):
//   * gj_solve_kernel  : Gauss-Jordan elimination with partial pivoting on [D | R] for a
//                        batch of small blocks (D up to 64 x 64): R = I gives D^-1 (the
//                        pivot-block inverse of the block LU), R = t_0 gives S_00^-1 t_0.
//   * build_m_kernel   : M = I - blockdiag(t) G.
//   * scale_kernel     : C = beta C (the k == 0 / alpha == 0 case of the GEMM API).
// These are the only places with O(n b^2) / O(n^2 b) binary64 arithmetic of the solve.
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

void launch_gj(const GjParams& p, int max_nb, int max_nrhs, int batch, cudaStream_t st) {
  const size_t smem = sizeof(double2) * static_cast<size_t>(max_nb) * (max_nb + max_nrhs);
  if (smem > 48 * 1024) cudaFuncSetAttribute(gj_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  gj_solve_kernel<<<batch, GJ_THREADS, smem, st>>>(p);
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

// Fill the per-solve tables of one step of the batched block LU (step >= 0), or of the final
// S_00^-1 t_0 solve (step < 0).  Step s eliminates J = [p, q) with q = n - s nb and
// p = max(q - nb, b), keeping R = [0, p); solves with q <= b are finished (sizes set to 0).
__global__ void kkr_step_kernel(int step, int nsolves, const int* __restrict__ n, double2* const* M, int b,
                                int nb, double2* dinv, KkrStep t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsolves) return;
  const int ni = n[i];
  double2* Mi = M[i];
  if (step < 0) {
    t.D[i] = Mi; t.ldd[i] = ni; t.nbv[i] = b;
    return;
  }
  const int q = ni - step * nb;
  if (q <= b) {
    t.nbv[i] = 0; t.m1[i] = 0; t.n1[i] = 0; t.k1[i] = 1; t.m2[i] = 0; t.n2[i] = 0; t.k2[i] = 1;
    t.D[i] = Mi; t.ldd[i] = ni; t.X[i] = dinv; t.ldx[i] = 1;
    t.A1[i] = Mi; t.lda1[i] = ni; t.B1[i] = dinv; t.ldb1[i] = 1; t.C1[i] = Mi; t.ldc1[i] = ni;
    t.A2[i] = Mi; t.lda2[i] = ni; t.B2[i] = Mi; t.ldb2[i] = ni; t.C2[i] = Mi; t.ldc2[i] = ni;
    return;
  }
  const int p = max(q - nb, b);
  const int w = q - p;
  double2* Di = dinv + static_cast<long long>(i) * nb * nb;
  t.D[i] = Mi + p + static_cast<long long>(p) * ni; t.ldd[i] = ni; t.nbv[i] = w; t.X[i] = Di; t.ldx[i] = w;
  double2* L = Mi + static_cast<long long>(p) * ni;
  t.A1[i] = L; t.lda1[i] = ni; t.B1[i] = Di; t.ldb1[i] = w; t.C1[i] = L; t.ldc1[i] = ni;
  t.m1[i] = p; t.n1[i] = w; t.k1[i] = w;
  t.A2[i] = L; t.lda2[i] = ni; t.B2[i] = Mi + p; t.ldb2[i] = ni; t.C2[i] = Mi; t.ldc2[i] = ni;
  t.m2[i] = p; t.n2[i] = p; t.k2[i] = w;
}

void launch_kkr_step(int step, int nsolves, const int* n, double2* const* M, int b, int nb, double2* dinv,
                     const KkrStep& t, cudaStream_t st) {
  kkr_step_kernel<<<(nsolves + 127) / 128, 128, 0, st>>>(step, nsolves, n, M, b, nb, dinv, t);
  record_launch();
}

}  // namespace ozk
