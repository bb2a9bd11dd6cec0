// Hermitian eigensolver of the mixed-precision Rayleigh-Ritz step (Algorithm 1 step 4 on the mixed path):
// an FP32 solve refined in FP64.
//
//  1. FP32: Householder tridiagonalisation in one CTA with the whole matrix in shared memory
//     (k_tridiag_cta), multisection, inverse iteration and back-transformation (the FP64 solver's kernels
//     instantiated for float). GB300 runs FP32 at 64x its FP64 rate, and the one-CTA reduction needs no
//     cluster or grid barriers.
//  2. FP64 refinement (one or two steps) of the eigenvector matrix X by the iteration of Ogita and Aishima (Japan J. Indust.
//     Appl. Math. 35, 2018, "Iterative refinement for symmetric eigenvalue decomposition"), written for
//     the Hermitian case: R = I - X^H X, S = X^H A X, lambda_i = S_ii / (1 - R_ii),
//     delta = 2 (||S - diag(lambda)|| + ||A|| ||R||); E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)
//     when lambda_i and lambda_j lie in different clusters (runs of eigenvalues closer than
//     max(delta, 1e-3 ||A||): no closer than the clusters of the FP32 inverse iteration, inside which the
//     vectors are only orthogonalised), E_ij = R_ij / 2 inside a cluster; X <- X + X E. Each step squares
//     the error of X across clusters.
//  3. Clusters of close eigenvalues are only orthonormalised by step 2; a Rayleigh-Ritz inside each
//     cluster (FP64 Jacobi on X_c^H A X_c) resolves them.
// The products are FP64 n x n complex GEMMs spread over many CTAs (k_zgemm16). Near convergence the
// refinement starts instead from the permutation that sorts the diagonal (a warm start) and keeps X in the
// form P (I + F), where every product is one of small matrices and runs in FP32 (k_fgemm16).
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "jacobi_small.cuh"
#include "paro_ctx.h"

namespace paro {

// pieces of the FP64 solver instantiated for float (k_eigh.cu)
template <typename R>
int invit(Ctx* c, int n, const R* d, const R* e, const R* w, R* Z, int* info);
int eigh_fp32_pieces(Ctx* c, int n, const float* d, const float* e, float* w, const float2* U, const float* tau,
                     const float2* ph, float* Z, float2* V, int* info);

static const int kMixMaxN = 160;  // largest n whose FP32 matrix fits one CTA's shared memory
// a pair whose refinement correction exceeds this joins one cluster (k_refine_lam), as long as no cluster
// grows beyond kCoupleMaxCluster columns; only while at least half of the last eight warm starts ended with a
// correction below 1e-5 (near convergence: far from it most pairs are coupled, and the FP32 solve is the
// faster route)
static const double kCouple = 1e-2;
static const int kCoupleMaxCluster = 8;

// ------------------------------------------------------------------------------------------------
// Householder tridiagonalisation, one CTA, matrix (FP32) in shared memory. The same reflectors and outputs
// as the FP64 kernels: u_j in U[j][0..m), tau, the complex off-diagonals ecx, d; then the phase diagonal D
// (D_0 = 1, D_{j+1} = D_j conj(e_j)/|e_j|) and the real off-diagonals |e_j|. Input a: full Hermitian FP64;
// only the lower triangle of the trailing matrix is kept current (the upper part is read as its conjugate).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tridiag_cta(int n, const double2* __restrict__ a, float2* __restrict__ U,
                                                      float* __restrict__ d, float* __restrict__ e,
                                                      float2* __restrict__ ph, float* __restrict__ tau,
                                                      float2* __restrict__ ecx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = n + 1;
  float2* A = reinterpret_cast<float2*>(smem_raw);  // n x ld
  float2* u = A + (size_t)n * ld;
  float2* w = u + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx - i * n;
    const double2 v = a[idx];
    A[i * ld + k] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1;
    // The reflector of column j, by every warp from the column in registers (FP32: the FP64 refinement
    // follows), so no barrier separates it from the matrix-vector product; lane holds u_k for
    // k = lane + 32 c (c < KC). Warp 0 also writes it to shared memory (read by the update) and out.
    constexpr int KC = (kMixMaxN + 31) / 32;
    float2 ur[KC];
    float nrm2 = 0.f;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const int k = lane + 32 * c;
      ur[c] = k < m ? A[(j + 1 + k) * ld + j] : make_float2(0.f, 0.f);
      nrm2 += ur[c].x * ur[c].x + ur[c].y * ur[c].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
    const float2 x0 = make_float2(__shfl_sync(0xffffffffu, ur[0].x, 0), __shfl_sync(0xffffffffu, ur[0].y, 0));
    const float ax0 = hypotf(x0.x, x0.y);
    const float nx = sqrtf(nrm2);
    float2 alpha = x0;
    float t = 0.f;
    if (m > 1 && nx > 0.f && nrm2 - ax0 * ax0 > 0.f) {
      const float2 phs = ax0 > 0.f ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.f, 0.f);
      alpha = make_float2(-phs.x * nx, -phs.y * nx);
      if (lane == 0) ur[0] = csub(x0, alpha);
      t = 1.f / (nrm2 + nx * ax0);
    }
    if (warp == 0) {
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int k = lane + 32 * c;
        if (k < m) {
          u[k] = ur[c];
          U[(size_t)j * n + k] = ur[c];
        }
      }
      if (lane == 0) {
        tau[j] = t;
        ecx[j] = alpha;
        d[j] = A[j * ld + j].x;
      }
    }
    if (t == 0.f) continue;  // the same in every warp: no barrier is skipped by some warps only
    // p_i = t sum_k B_ik u_k (B_ik = conj(B_ki) above the diagonal): rows i and i + nwarp together, so that
    // the two 32-lane reductions overlap
    for (int i0 = warp; i0 < m; i0 += 2 * nwarp) {
      const int i1 = i0 + nwarp;
      const bool has1 = i1 < m;
      const float2* row0 = A + (j + 1 + i0) * ld + (j + 1);
      const float2* col0 = A + (j + 1) * ld + (j + 1 + i0);
      const float2* row1 = A + (j + 1 + (has1 ? i1 : i0)) * ld + (j + 1);
      const float2* col1 = A + (j + 1) * ld + (j + 1 + (has1 ? i1 : i0));
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int k = lane + 32 * c;
        if (k < m) {
          float2 b0, b1;
          if (k <= i0) {
            b0 = row0[k];
          } else {
            b0 = col0[k * ld];
            b0.y = -b0.y;
          }
          if (k <= i1) {
            b1 = row1[k];
          } else {
            b1 = col1[k * ld];
            b1.y = -b1.y;
          }
          a0.x = fmaf(b0.x, ur[c].x, fmaf(-b0.y, ur[c].y, a0.x));
          a0.y = fmaf(b0.x, ur[c].y, fmaf(b0.y, ur[c].x, a0.y));
          a1.x = fmaf(b1.x, ur[c].x, fmaf(-b1.y, ur[c].y, a1.x));
          a1.y = fmaf(b1.x, ur[c].y, fmaf(b1.y, ur[c].x, a1.y));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o);
        a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o);
        a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
        a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
      }
      if (lane == 0) {
        w[i0] = make_float2(t * a0.x, t * a0.y);
        if (has1) w[i1] = make_float2(t * a1.x, t * a1.y);
      }
    }
    __syncthreads();
    // every warp: K = (t/2) u^H p (real), w = p - K u in registers (no second barrier for w)
    float2 wr[KC];
    float kre = 0.f;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const int k = lane + 32 * c;
      wr[c] = k < m ? w[k] : make_float2(0.f, 0.f);
      kre += ur[c].x * wr[c].x + ur[c].y * wr[c].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kre += __shfl_xor_sync(0xffffffffu, kre, o);
    const float K = 0.5f * t * kre;
#pragma unroll
    for (int c = 0; c < KC; ++c) wr[c] = make_float2(wr[c].x - K * ur[c].x, wr[c].y - K * ur[c].y);
    for (int i = warp; i < m; i += nwarp) {  // B -= u w^H + w u^H on and below the diagonal, one row per warp
      const float2 ui = u[i], pi = w[i];
      const float2 wi = make_float2(pi.x - K * ui.x, pi.y - K * ui.y);
      float2* row = A + (j + 1 + i) * ld + (j + 1);
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int k = lane + 32 * c;
        if (k <= i) {
          const float2 uk = ur[c], wk = wr[c];
          float2 bv = row[k];
          bv.x -= ui.x * wk.x + ui.y * wk.y + wi.x * uk.x + wi.y * uk.y;
          bv.y -= ui.y * wk.x - ui.x * wk.y + wi.y * uk.x - wi.x * uk.y;
          row[k] = bv;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    d[n - 1] = A[(n - 1) * ld + (n - 1)].x;
    ph[0] = make_float2(1.f, 0.f);
    for (int j = 0; j + 1 < n; ++j) {
      const float v = hypotf(ecx[j].x, ecx[j].y);
      e[j] = v;
      ph[j + 1] = v > 0.f ? cmul(ph[j], make_float2(ecx[j].x / v, -ecx[j].y / v)) : ph[j];
    }
    e[n - 1] = 0.f;
  }
}

// ------------------------------------------------------------------------------------------------
// FP64 n x n complex products: part[z] = op(A) B over the K slice z (op = identity, or conjugate transpose
// when ah); 16 x 16 outputs per CTA. k_zreduce sums the slices in order: C = sum (+ C when add).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_zgemm16(int n, const double2* __restrict__ A, int ah,
                                                 const double2* __restrict__ B, double2* __restrict__ part,
                                                 int kslice) {
  __shared__ double2 As[16][17], Bs[16][17];
  if (ah > 1 && blockIdx.y < blockIdx.x) return;  // Hermitian result: tiles on and below the diagonal
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  const int k0 = blockIdx.z * kslice, k1 = min(n, k0 + kslice);
  double2 acc = make_double2(0.0, 0.0);
  for (int kk = k0; kk < k1; kk += 16) {
    const int ia = i0 + ty, ka = kk + tx;
    double2 av = make_double2(0.0, 0.0);
    if (ia < n && ka < k1) av = ah ? cconj(A[(size_t)ka * n + ia]) : A[(size_t)ia * n + ka];
    As[ty][tx] = av;
    const int kb = kk + ty, jb = j0 + tx;
    Bs[ty][tx] = (kb < k1 && jb < n) ? B[(size_t)kb * n + jb] : make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
      const double2 x = As[ty][k], y = Bs[k][tx];
      acc.x = fma(x.x, y.x, fma(-x.y, y.y, acc.x));
      acc.y = fma(x.x, y.y, fma(x.y, y.x, acc.y));
    }
    __syncthreads();
  }
  const int i = i0 + ty, jj = j0 + tx;
  if (i < n && jj < n) part[(size_t)blockIdx.z * n * n + (size_t)i * n + jj] = acc;
}

// nrm (optional, one float per CTA of 256 threads): the CTA's sum of |C_ij - d_ij|^2 over i != j plus, when
// unit, |C_ii - 1|^2 on the diagonal (in FP32: it only sets the refinement's cluster threshold)
__global__ void __launch_bounds__(256) k_zreduce(int n, int nz, const double2* __restrict__ part,
                                                 double2* __restrict__ C, int add, int herm,
                                                 float* __restrict__ nrm, int unit) {
  __shared__ float red[32];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (idx < n * n) {
    const int i = idx / n, j = idx - i * n;
    const bool mirror = herm && (i >> 4) < (j >> 4);  // tile above the diagonal: conj of the (j, i) sum
    const size_t src = mirror ? (size_t)j * n + i : (size_t)idx;
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < nz; ++z) s = cadd(s, part[(size_t)z * n * n + src]);
    if (mirror) s = cconj(s);
    if (add) s = cadd(C[idx], s);
    C[idx] = s;
    if (nrm && (i != j || unit)) {
      const float x = (float)(i == j ? s.x - 1.0 : s.x), y = (float)s.y;
      e = x * x + y * y;
    }
  }
  if (nrm) {
    e = block_sumf(e, red);
    if (threadIdx.x == 0) nrm[blockIdx.x] = e;
  }
}

// ------------------------------------------------------------------------------------------------
// One refinement step's small quantities. k_refine_lam (one CTA): lambda_i = S_ii / G_ii, delta and the
// clusters (cl: cluster index per column; cst: first column of each cluster; ncl). delta only sets the
// cluster threshold, so its norms are summed in FP32 (no FP64 pipe on the n^2 sweep).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_refine_lam(int n, const double2* __restrict__ G,
                                                     const double2* __restrict__ S, const float* __restrict__ nrm,
                                                     int nnrm, double* __restrict__ lam, int* __restrict__ cl,
                                                     int* __restrict__ cst, int* __restrict__ ncl,
                                                     float* __restrict__ emax, double couple,
                                                     const float2* __restrict__ S32, const float2* __restrict__ Gm32) {
  __shared__ float red[32];
  __shared__ double s_lam[kMixMaxN];
  __shared__ int s_reach[kMixMaxN], s_cl[kMixMaxN], s_cst[kMixMaxN + 1];
  __shared__ int s_wc[32], s_ncl, s_long;
  __shared__ double s_delta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) {
    const double l = S[(size_t)i * n + i].x / G[(size_t)i * n + i].x;
    lam[i] = l;
    s_lam[i] = l;
  }
  // ||S - diag||_F^2 (off-diagonal part) and ||I - G||_F^2 from the per-CTA sums of k_zreduce
  float ns = 0.f, nr = 0.f, na = 0.f;
  for (int b = tid; b < nnrm; b += blockDim.x) {
    nr += nrm[b];
    ns += nrm[nnrm + b];
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) na = fmaxf(na, fabsf((float)s_lam[i]));
  ns = block_sumf(ns, red);
  __syncthreads();
  nr = block_sumf(nr, red);
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) na = fmaxf(na, __shfl_xor_sync(0xffffffffu, na, o));
  if (lane == 0) red[warp] = na;
  __syncthreads();
  if (tid == 0) {
    float mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    // clusters: at least the FP32 solver's own (eigenvalues closer than 1e-3 ||A||, whose vectors inverse
    // iteration only orthogonalised), so that every pair corrected below is already accurate to first order
    s_delta = fmax(2.0 * ((double)sqrtf(ns) + (double)mx * (double)sqrtf(nr)), 1e-3 * (double)mx);
  }
  __syncthreads();
  // Pairs whose correction would not be small, |S_ij + lambda_j R_ij| > couple |lambda_j - lambda_i| (a pair
  // of close eigenvalues that the potential's change has mixed), join one cluster: the Rayleigh-Ritz inside
  // the cluster resolves them exactly, where the refinement would need several steps. Pairs up to 32 columns
  // apart; reach[i] = the last column coupled to i.
  for (int i = warp; i < n; i += (int)(blockDim.x >> 5)) {
    int r = i;
    const int j = i + 1 + lane;
    if (couple > 0.0 && j < n) {  // in FP32 (a threshold test) from the FP32 copies of S and G - I
      const float2 g = Gm32 ? Gm32[(size_t)i * n + j] : make_float2(0.f, 0.f), sv = S32[(size_t)i * n + j];
      const float lj = (float)s_lam[j];
      const float nx = sv.x - lj * g.x, ny = sv.y - lj * g.y;  // S_ij + lambda_j R_ij with R = I - G (i != j)
      const float gap = lj - (float)s_lam[i], cf = (float)couple;
      if (nx * nx + ny * ny > cf * cf * gap * gap) r = j;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) s_reach[i] = r;
  }
  __syncthreads();
  // inclusive prefix maximum of reach (Hillis-Steele)
  for (int off = 1; off < n; off <<= 1) {
    const int v = (tid < n && tid >= off) ? s_reach[tid - off] : 0;
    __syncthreads();
    if (tid < n && tid >= off) s_reach[tid] = max(s_reach[tid], v);
    __syncthreads();
  }
  // A new cluster starts at i when lambda_i - lambda_{i-1} > delta and no coupled pair spans i (prefix reach
  // below i); cluster index = inclusive count of starts up to i (ballot within a warp, then the warps' counts
  // in order). Without the coupled pairs when they would make a cluster longer than kCoupleMaxCluster
  // columns: far from convergence most pairs are coupled, and one large cluster would turn the warm start
  // into a Jacobi diagonalisation in FP64 (the FP32 solve is faster there).
  const int nw = (n + 31) / 32;
  for (int pass = 0; pass < 2; ++pass) {
    const bool start = tid < n && tid > 0 && s_lam[tid] - s_lam[tid - 1] > s_delta &&
                       (pass == 1 || s_reach[tid - 1] < tid);
    const unsigned bal = warp < nw ? __ballot_sync(0xffffffffu, start) : 0u;
    if (warp < nw && lane == 0) s_wc[warp] = __popc(bal);
    if (tid == 0) s_long = 0;
    __syncthreads();
    if (tid < n) {
      int cidx = __popc(bal & (0xffffffffu >> (31 - lane)));
      for (int w = 0; w < warp; ++w) cidx += s_wc[w];
      s_cl[tid] = cidx;
      if (tid == 0 || start) s_cst[cidx] = tid;
      if (tid == n - 1) {
        s_cst[cidx + 1] = n;
        s_ncl = cidx + 1;
      }
    }
    __syncthreads();
    if (tid < s_ncl && s_cst[tid + 1] - s_cst[tid] > kCoupleMaxCluster) s_long = 1;
    __syncthreads();
    if (!s_long) break;
  }
  for (int i = tid; i < n; i += blockDim.x) cl[i] = s_cl[i];
  for (int i = tid; i <= s_ncl; i += blockDim.x) cst[i] = s_cst[i];
  if (tid == 0) {
    *ncl = s_ncl;
    if (emax) *emax = 0.f;
  }
}

// E (many CTAs): R = I - G; E_ij = R_ij / 2 inside a cluster, else (S_ij + lambda_j R_ij) / (lambda_j -
// lambda_i). E is a correction of size ~ the FP32 solver's error, so the quotient is formed in FP32 from
// an FP64 numerator and difference: its relative FP32 rounding is far below what the step needs.
// emax (may be null; zeroed by k_refine_lam): the largest |Re E_ij|, |Im E_ij| (the warm start's convergence
// test), by one atomic maximum per CTA on the float's bits (non-negative floats order as their bits)
__global__ void __launch_bounds__(256) k_refine_e(int n, const double2* __restrict__ G, const double2* __restrict__ S,
                                                  const double* __restrict__ lam, const int* __restrict__ cl,
                                                  double2* __restrict__ E, float* __restrict__ emax,
                                                  float2* __restrict__ E32) {
  __shared__ float red[32];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.f;
  if (idx < n * n) {
    const int i = idx / n, j = idx - i * n;
    double2 rv = cscale(G[idx], -1.0);
    if (i == j) rv.x += 1.0;
    double2 e;
    if (cl[i] == cl[j]) {
      e = cscale(rv, 0.5);
    } else {
      const double lj = lam[j];
      const double2 num = make_double2(fma(lj, rv.x, S[idx].x), fma(lj, rv.y, S[idx].y));
      const float inv = 1.0f / (float)(lj - lam[i]);
      e = make_double2((double)((float)num.x * inv), (double)((float)num.y * inv));
    }
    E[idx] = e;
    const float2 ef = make_float2((float)e.x, (float)e.y);
    if (E32) E32[idx] = ef;
    m = fmaxf(fabsf(ef.x), fabsf(ef.y));
  }
  if (!emax) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(reinterpret_cast<int*>(emax), __float_as_int(m));
  }
}

// S_ij = x_i^H (A x_j) = sum_r conj(X[r][i]) T1[r][j] for the pairs (i, j) of one cluster only: the
// Rayleigh-Ritz inside the clusters (and lambda of singletons) reads nothing else of S
// one warp per pair (i, j), lanes over r
__global__ void k_blockdiag_xhat(int n, const double2* __restrict__ X, const double2* __restrict__ T1,
                                 const int* __restrict__ cl, double2* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  if (cl[i] != cl[j]) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int r = lane; r < n; r += 32) acc = cadd(acc, cmul(cconj(X[(size_t)r * n + i]), T1[(size_t)r * n + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) S[idx] = acc;
}

// Rayleigh-Ritz inside each cluster of two or more columns: S_c = (X^H A X)_cc (k x k, k <= 64)
// diagonalised by Jacobi, X_c <- X_c Q, lam_c = its eigenvalues; one CTA per cluster. Singleton
// clusters take lam_i = S_ii. info |= 4 for a cluster larger than 64, |= 8 if Jacobi did not converge.
__global__ void __launch_bounds__(256) k_cluster_rr(int n, const double2* __restrict__ S, const int* __restrict__ cst,
                                                    const int* __restrict__ ncl, double2* __restrict__ X,
                                                    double* __restrict__ lam, int* __restrict__ info) {
  constexpr int KM = 64, LD = KM + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Am = reinterpret_cast<double2*>(smem_raw);
  double2* Vm = Am + KM * LD;
  __shared__ int pos[KM];
  __shared__ double rc[KM / 2], rs[KM / 2];
  __shared__ double2 rph[KM / 2];
  __shared__ int rp[KM / 2], rq[KM / 2];
  __shared__ double red[32];
  __shared__ double s_off, s_tot;
  const int c = blockIdx.x;
  if (c >= *ncl) return;
  const int c0 = cst[c], k = cst[c + 1] - c0;
  if (k == 1) {
    if (threadIdx.x == 0) lam[c0] = S[(size_t)c0 * n + c0].x;
    return;
  }
  if (k > KM) {
    if (threadIdx.x == 0) atomicOr(info, 4);
    return;
  }
  if (k == 2) {  // a pair (the common cluster: a degenerate level split by the potential) in closed form
    __shared__ double2 q[4];
    if (threadIdx.x == 0) {
      // [[a, b], [conj b, d]] = D [[a, beta], [beta, d]] D^H with b = beta phi, D = diag(1, conj phi); the
      // real matrix turns by theta = atan2(2 beta, a - d) / 2 to diag(m + r, m - r)
      const double a = S[(size_t)c0 * n + c0].x, d = S[(size_t)(c0 + 1) * n + c0 + 1].x;
      const double2 b = S[(size_t)c0 * n + c0 + 1];
      const double beta = hypot(b.x, b.y);
      const double2 phc = beta > 0.0 ? make_double2(b.x / beta, -b.y / beta) : make_double2(1.0, 0.0);
      const double th = 0.5 * atan2(2.0 * beta, a - d), cs = cos(th), sn = sin(th);
      const double m = 0.5 * (a + d), r = hypot(0.5 * (a - d), beta);
      q[0] = make_double2(cs, 0.0);                   // Q_00
      q[1] = make_double2(-sn, 0.0);                  // Q_01
      q[2] = make_double2(phc.x * sn, phc.y * sn);    // Q_10
      q[3] = make_double2(phc.x * cs, phc.y * cs);    // Q_11
      lam[c0] = m + r;
      lam[c0 + 1] = m - r;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double2 x0 = X[(size_t)i * n + c0], x1 = X[(size_t)i * n + c0 + 1];
      X[(size_t)i * n + c0] = cadd(cmul(x0, q[0]), cmul(x1, q[2]));
      X[(size_t)i * n + c0 + 1] = cadd(cmul(x0, q[1]), cmul(x1, q[3]));
    }
    return;
  }
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx - i * k;
    Am[i * LD + j] = S[(size_t)(c0 + i) * n + (c0 + j)];
    Vm[i * LD + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  JacobiScratch sc{pos, rc, rs, rph, rp, rq, red, &s_off, &s_tot};
  const int ok = jacobi_herm(k, LD, Am, Vm, sc);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) lam[c0 + j] = Am[j * LD + j].x;
  // X_c <- X_c Q: each thread one row at a time (k <= 64 values in registers)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double2 row[KM];
    for (int l = 0; l < k; ++l) row[l] = X[(size_t)i * n + c0 + l];
    for (int j = 0; j < k; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int l = 0; l < k; ++l) s = cadd(s, cmul(row[l], Vm[l * LD + j]));
      X[(size_t)i * n + c0 + j] = s;
    }
  }
  if (threadIdx.x == 0 && !ok) atomicOr(info, 8);
}

// ascending order (ties by index): w[j] = lam[perm j], V[:, j] = X[:, perm j]
// a 64-bit integer that orders as the double does (sign and magnitude bits turned into a two's complement
// order): the sorting counts compare these on the integer pipe, where GB300's FP64 compares would take the
// slow FP64 pipe
__device__ __forceinline__ long long order_key(double d) {
  const long long b = __double_as_longlong(d);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// (n <= 1024: the eigenvalues' order keys are staged in shared memory)
__global__ void k_eig_sort(int n, const double* __restrict__ lam, const double2* __restrict__ X, double* __restrict__ w,
                           double2* __restrict__ V, int* __restrict__ perm) {
  __shared__ long long s_l[1024];
  for (int j = threadIdx.x; j < n; j += blockDim.x) s_l[j] = order_key(lam[j]);
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < n) {
    const long long a = s_l[tid];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const long long b = s_l[j];
      r += (b < a) || (b == a && j < tid);
    }
    perm[r] = tid;
  }
}

// rank (may be null): X holds P^H times the vectors (the warm start's permuted rows): V[i][:] = X[rank(i)][:]
__global__ void k_eig_permute(int n, const double* __restrict__ lam, const double2* __restrict__ X,
                              const int* __restrict__ perm, const int* __restrict__ rank, double* __restrict__ w,
                              double2* __restrict__ V) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  V[idx] = X[(size_t)(rank ? rank[i] : i) * n + perm[j]];
  if (i == 0) w[j] = lam[perm[j]];
}

__global__ void k_f2d(int n, const float2* __restrict__ a, double2* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

__global__ void k_herm_full_mixed(int n, const double2* __restrict__ Ain, double2* __restrict__ A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  A[idx] = (i >= j) ? Ain[idx] : cconj(Ain[(size_t)j * n + i]);
}

// C = op(A) B (+ C), n x n FP64. herm: the result is Hermitian (A^H A, or A^H M A with B = M A), so only
// the tiles on and below the diagonal are computed and the rest mirrored.
static int zgemm(Ctx* c, int n, const double2* A, bool ah, const double2* B, double2* C, bool add, double2* part,
                 bool herm = false, float* nrm = nullptr, bool unit = false) {
  const int nz = std::max(1, std::min(8, (n + 47) / 48));
  const int kslice = ((n + nz - 1) / nz + 15) / 16 * 16;
  const int z = (n + kslice - 1) / kslice;
  const int t = (n + 15) / 16;
  cudaEvent_t ev = prof_begin(c);
  k_zgemm16<<<dim3(t, t, z), 256, 0, c->stream>>>(n, A, ah ? (herm ? 2 : 1) : 0, B, part, kslice);
  PARO_LAUNCH(c, "k_zgemm16");
  k_zreduce<<<(n * n + 255) / 256, 256, 0, c->stream>>>(n, z, part, C, add ? 1 : 0, herm ? 1 : 0, nrm,
                                                        unit ? 1 : 0);
  prof_end(c, "zgemm", ev);
  PARO_LAUNCH(c, "k_zreduce");
  return PARO_OK;
}

// Warm start of the refinement: X0 = the permutation that sorts the diagonal of A, X0[i][rank(i)] = 1 with
// rank(i) = #{j : a_jj < a_ii, or a_jj = a_ii and j < i}; at_rank is its inverse (one CTA, n <= 1024)
__global__ void k_warm_perm(int n, const double2* __restrict__ A, int* __restrict__ rank, int* __restrict__ at_rank) {
  __shared__ long long s_d[1024];
  const int i = threadIdx.x;
  if (i < n) s_d[i] = order_key(A[(size_t)i * n + i].x);
  __syncthreads();
  if (i >= n) return;
  const long long d = s_d[i];
  int r = 0;
  for (int j = 0; j < n; ++j) {
    const long long e = s_d[j];
    r += (e < d || (e == d && j < i)) ? 1 : 0;
  }
  rank[i] = r;
  at_rank[r] = i;
}

// The first refinement step from X0 needs no products: G = X0^H X0 = I and S = X0^H A X0 = A with rows and
// columns in rank order (A given by its lower triangle); N32: the off-diagonal part of S in FP32. nrm as
// k_zreduce leaves it for the pair (G, S): per CTA of 256 entries, zero for G and the off-diagonal sum of
// |S_ij|^2 for S.
__global__ void __launch_bounds__(256) k_warm_s(int n, const double2* __restrict__ A, const int* __restrict__ at_rank,
                                                double2* __restrict__ G, double2* __restrict__ S,
                                                float* __restrict__ nrm, int nnrm, float2* __restrict__ N32) {
  __shared__ float red[32];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (idx < n * n) {
    const int r = idx / n, q = idx - r * n, i = at_rank[r], j = at_rank[q];
    const double2 v = i >= j ? A[(size_t)i * n + j] : cconj(A[(size_t)j * n + i]);  // A: its lower triangle
    S[idx] = v;
    G[idx] = make_double2(r == q ? 1.0 : 0.0, 0.0);
    const float x = (float)v.x, y = (float)v.y;
    N32[idx] = r != q ? make_float2(x, y) : make_float2(0.f, 0.f);  // N, the off-diagonal part, in FP32
    if (r != q) e = x * x + y * y;
  }
  e = block_sumf(e, red);
  if (threadIdx.x == 0) {
    nrm[blockIdx.x] = 0.f;
    nrm[nnrm + blockIdx.x] = e;
  }
}

// X1 = X0 (I + E): row i of X1 is row rank(i) of I + E
__global__ void k_warm_x1(int n, const int* __restrict__ rank, const double2* __restrict__ E, double2* __restrict__ X) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n, r = rank[i];
  double2 v = E[(size_t)r * n + j];
  if (r == j) v.x += 1.0;
  X[idx] = v;
}

// ------------------------------------------------------------------------------------------------
// Warm-start refinement in the form X = P (I + F): P the permutation that sorts the diagonal, A' = P^H A P
// (exact, FP64) and F the accumulated correction, small near convergence. Then
//   X^H X     = I + F + F^H + F^H F,
//   X^H A X   = A' + A'F + (A'F)^H + F^H (A'F),
//   X (I + E) = P (I + F + E + F E),
// and with A' = D + N (D its diagonal, N the off-diagonal part, of the size of the residuals) every
// product that remains, N F, F^H F, F^H (A'F) and F E, is one of small quantities: rounded in FP32 its
// error is ~1e-7 of a product that is itself far below 1, so these products run on the FP32 pipe, and
// only the exact parts (I, D F, A') are added in FP64. (GB300's FP64 rate is 1/64 of its FP32 rate.)
// ------------------------------------------------------------------------------------------------
struct FProd {
  const float2* A32;  // the operands of the FP32 product (n x n, row-major; FP32 copies)
  const float2* B32;
  const double2* A;   // the same in FP64, for the epilogue terms (may be null when no term reads them)
  const double2* B;
  double2* C;
  float2* C32;  // (may be null) an FP32 copy of the result, for the next product
  int ah;       // op(A) = A^H
  int diag;     // leave the k = i term out of the FP32 sum and add A_ii B_ij in FP64 (A' F as D F + N F)
  int add_a;    // add op(A)_ij to the result
  int add_ab;   // add A_ij + B_ij to the result (F + E + F E)
  double2* xp;  // (may be null) also I + B into xp (X' = I + F beside T1 = A' X')
};

// C = op(A) B (+ the epilogue terms) for one or two products (blockIdx.z), 16 x 16 outputs per CTA (n <=
// kMixMaxN): the CTA's 16 rows of op(A) and 16 columns of B are staged whole in shared memory from the
// operands' FP32 copies (one round of loads, no conversions), then FP32 products, the partial sum of every
// 16 terms added into an FP32 two-sum pair; FP64 only in the epilogue (GB300's FP64 pipe, conversions
// included, runs at 1/64 of the FP32 rate)
__global__ void __launch_bounds__(256) k_fgemm16(int n, FProd p0, FProd p1) {
  __shared__ float2 As[16][kMixMaxN + 1], Bs[kMixMaxN][17];
  const FProd& p = blockIdx.z ? p1 : p0;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  const int i = i0 + ty, j = j0 + tx;
  const int n16 = (n + 15) & ~15;
  for (int idx = threadIdx.x; idx < 16 * n16; idx += blockDim.x) {
    int r, k;
    if (p.ah) {  // op(A)_ik = conj(A_ki): consecutive threads along i
      r = idx & 15;
      k = idx >> 4;
    } else {
      r = idx / n16;
      k = idx - r * n16;
    }
    const int ia = i0 + r;
    float2 av = make_float2(0.f, 0.f);
    if (ia < n && k < n && !(p.diag && ia == k)) {
      av = p.ah ? p.A32[(size_t)k * n + ia] : p.A32[(size_t)ia * n + k];
      if (p.ah) av.y = -av.y;
    }
    As[r][k] = av;
  }
  for (int idx = threadIdx.x; idx < 16 * n16; idx += blockDim.x) {
    const int k = idx >> 4, cc = idx & 15, jb = j0 + cc;
    Bs[k][cc] = (k < n && jb < n) ? p.B32[(size_t)k * n + jb] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
  for (int kk = 0; kk < n16; kk += 16) {
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 x = As[ty][kk + k], y = Bs[kk + k][tx];
      sx = fmaf(x.x, y.x, fmaf(-x.y, y.y, sx));
      sy = fmaf(x.x, y.y, fmaf(x.y, y.x, sy));
    }
    two_sum_acc(hx, lx, sx);
    two_sum_acc(hy, ly, sy);
  }
  if (i >= n || j >= n) return;
  double2 acc = make_double2((double)hx + (double)lx, (double)hy + (double)ly);
  if (p.diag) {  // A_ii B_ij in FP64 (op(A)_ii = conj(A_ii) when ah)
    double2 d = p.A[(size_t)i * n + i];
    if (p.ah) d = cconj(d);
    acc = cadd(acc, cmul(d, p.B[(size_t)i * n + j]));
  }
  if (p.add_a) acc = cadd(acc, p.ah ? cconj(p.A[(size_t)j * n + i]) : p.A[(size_t)i * n + j]);
  if (p.add_ab) acc = cadd(acc, cadd(p.A[(size_t)i * n + j], p.B[(size_t)i * n + j]));
  p.C[(size_t)i * n + j] = acc;
  if (p.C32) p.C32[(size_t)i * n + j] = make_float2((float)acc.x, (float)acc.y);
  if (p.xp) {
    double2 x = p.B[(size_t)i * n + j];
    if (i == j) x.x += 1.0;
    p.xp[(size_t)i * n + j] = x;
  }
}

// G = I + F + F^H + FF and S = A' + AF + AF^H + FAF (and FP32 copies of G - I and S for the coupling test),
// with the per-CTA sums of k_zreduce for the cluster threshold: nrm[b] = sum |G_ij - d_ij|^2,
// nrm[nnrm + b] = sum over i != j of |S_ij|^2
__global__ void __launch_bounds__(256) k_fassemble(int n, const double2* __restrict__ Ap, const double2* __restrict__ F,
                                                   const double2* __restrict__ AF, const double2* __restrict__ FF,
                                                   const double2* __restrict__ FAF, double2* __restrict__ G,
                                                   double2* __restrict__ S, float* __restrict__ nrm, int nnrm,
                                                   float2* __restrict__ S32, float2* __restrict__ Gm32) {
  __shared__ float red[32];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float eg = 0.f, es = 0.f;
  if (idx < n * n) {
    const int i = idx / n, j = idx - i * n;
    const size_t t = (size_t)j * n + i;
    const double2 r = cadd(cadd(F[idx], cconj(F[t])), FF[idx]);  // G - I
    G[idx] = make_double2(r.x + (i == j ? 1.0 : 0.0), r.y);
    const double2 s = cadd(cadd(Ap[idx], cadd(AF[idx], cconj(AF[t]))), FAF[idx]);
    S[idx] = s;
    const float2 rf = make_float2((float)r.x, (float)r.y), sf = make_float2((float)s.x, (float)s.y);
    Gm32[idx] = rf;
    S32[idx] = sf;
    eg = rf.x * rf.x + rf.y * rf.y;
    if (i != j) es = sf.x * sf.x + sf.y * sf.y;
  }
  eg = block_sumf(eg, red);
  __syncthreads();
  es = block_sumf(es, red);
  if (threadIdx.x == 0) {
    nrm[blockIdx.x] = eg;
    nrm[nnrm + blockIdx.x] = es;
  }
}

static int fgemm(Ctx* c, int n, const FProd& p0, const FProd* p1) {
  const int t = (n + 15) / 16;
  k_fgemm16<<<dim3(t, t, p1 ? 2 : 1), 256, 0, c->stream>>>(n, p0, p1 ? *p1 : p0);
  PARO_LAUNCH(c, "k_fgemm16");
  return PARO_OK;
}

static int eigh_finish(Ctx* c, int n, const double2* a, const double2* Af, double2* X, double2* T1, double2* S,
                       double2* part, const int* cl, const int* cst, const int* ncl, double* lam, double* w,
                       double2* v, int* perm, int* info, bool clusters, const int** info_out);
static int eigh_finish_tail(Ctx* c, int n, const double2* a, double2* X, const double2* S, const int* cst,
                            const int* ncl, double* lam, double* w, double2* v, int* perm, int* info,
                            const int** info_out, const int* rank);

// warm-start bookkeeping: accepted when the last correction is below 1e-4 (the remaining error is of its
// square); after a failure the FP32 solve runs for the next 1, 2, 4, then 8 calls after consecutive failures
// (far from convergence the warm start keeps failing; near it a failure is a passing pair of close
// eigenvalues, and the next step usually succeeds)
static bool warm_outcome(Ctx* c, float emax) {
  c->eig_warm_last = emax;
  c->eig_warm_hist = ((c->eig_warm_hist << 1) | (emax < 1e-5f ? 1u : 0u)) & 0xffu;
  if (emax < 1e-4f) {
    c->eig_warm_fails = 0;
    return true;
  }
  c->eig_warm_skip = std::min(8, 1 << std::min(c->eig_warm_fails, 3)) - 1;
  ++c->eig_warm_fails;
  return false;
}

bool eigh_mixed_accept(Ctx* c, float emax) { return warm_outcome(c, emax); }

int eigh_mixed(Ctx* c, int n, const double2* a, double* w, double2* v, int refine_steps, bool warm,
               const int** info_out, const float** emax_out) {
  if (info_out) *info_out = nullptr;
  if (emax_out) *emax_out = nullptr;
  if (n < 2 || n > kMixMaxN) return eigh(c, n, a, w, v);
  const size_t nn = (size_t)n * n;
  double2* Af = static_cast<double2*>(ws_get(c, "em_A", nn * sizeof(double2)));
  double2* X = static_cast<double2*>(ws_get(c, "em_X", nn * sizeof(double2)));
  double2* T1 = static_cast<double2*>(ws_get(c, "em_T1", nn * sizeof(double2)));
  double2* G = static_cast<double2*>(ws_get(c, "em_G", nn * sizeof(double2)));
  double2* S = static_cast<double2*>(ws_get(c, "em_S", nn * sizeof(double2)));
  double2* part = static_cast<double2*>(ws_get(c, "em_part", 8 * nn * sizeof(double2)));
  float2* U32 = static_cast<float2*>(ws_get(c, "em_U32", nn * sizeof(float2)));
  float2* V32 = static_cast<float2*>(ws_get(c, "em_V32", nn * sizeof(float2)));
  float* Z32 = static_cast<float*>(ws_get(c, "em_Z32", nn * sizeof(float)));
  float* r32 = static_cast<float*>(ws_get(c, "em_r32", (size_t)6 * n * sizeof(float)));
  const int nnrm = (int)((nn + 255) / 256);  // per-CTA norm sums of G and of S, for the cluster threshold
  float* nrm = static_cast<float*>(ws_get(c, "em_nrm", (size_t)2 * nnrm * sizeof(float)));
  if (!nrm) return PARO_ERR_CUDA;
  double* lam = static_cast<double*>(ws_get(c, "em_lam", (size_t)n * sizeof(double)));
  int* ib = static_cast<int*>(ws_get(c, "em_int", (size_t)(3 * n + 8) * sizeof(int)));
  if (!Af || !X || !T1 || !G || !S || !part || !U32 || !V32 || !Z32 || !r32 || !lam || !ib) return PARO_ERR_CUDA;
  float *d32 = r32, *e32 = r32 + n, *tau32 = r32 + 2 * n, *w32 = r32 + 3 * n;
  float2* c32 = reinterpret_cast<float2*>(r32 + 4 * n);  // ph (n) then ecx: 2n floats each
  float2* ph32 = c32;
  int *cl = ib, *cst = ib + n, *perm = ib + 2 * n + 1, *flags = ib + 3 * n + 2;
  int* ncl = flags + 1;
  int* info = flags + 2;
  float2* ecx32 = static_cast<float2*>(ws_get(c, "em_ecx32", (size_t)n * sizeof(float2)));
  if (!ecx32) return PARO_ERR_CUDA;
  PARO_CU(c, cudaMemsetAsync(flags, 0, 6 * sizeof(int), c->stream));
  int st;
  // Rayleigh-Ritz near convergence: the matrix of a basis that already is close to the eigenvectors is
  // nearly diagonal, and two (or three) refinement steps from the permutation that sorts its diagonal reach
  // the accuracy one step gives from the FP32 eigenvectors; accepted when the last correction is below
  // 1e-4 (the remaining error is of its square), else the FP32 solve below runs
  if (warm && c->eig_warm_skip > 0) {
    --c->eig_warm_skip;
  } else if (warm) {
    cudaEvent_t evw = prof_begin(c);
    int* rk = static_cast<int*>(ws_get(c, "em_rank", (size_t)2 * n * sizeof(int)));
    double2* Ap = static_cast<double2*>(ws_get(c, "em_Ap", nn * sizeof(double2)));
    double2* F = static_cast<double2*>(ws_get(c, "em_F0", nn * sizeof(double2)));
    double2* Fn = static_cast<double2*>(ws_get(c, "em_F1", nn * sizeof(double2)));
    double2* AF = static_cast<double2*>(ws_get(c, "em_AF", nn * sizeof(double2)));
    double2* FF = static_cast<double2*>(ws_get(c, "em_FF", nn * sizeof(double2)));
    double2* FAF = static_cast<double2*>(ws_get(c, "em_FAF", nn * sizeof(double2)));
    // FP32 copies: N (off-diagonal part of A'), F and the next F, A'F, E, S and G - I
    float2* f32 = static_cast<float2*>(ws_get(c, "em_f32", 7 * nn * sizeof(float2)));
    if (!rk || !Ap || !F || !Fn || !AF || !FF || !FAF || !f32) return PARO_ERR_CUDA;
    float2 *N32 = f32, *F32 = f32 + nn, *Fn32 = f32 + 2 * nn, *AF32 = f32 + 3 * nn, *E32 = f32 + 4 * nn,
           *S32 = f32 + 5 * nn, *Gm32 = f32 + 6 * nn;
    k_warm_perm<<<1, 1024, 0, c->stream>>>(n, a, rk, rk + n);
    PARO_LAUNCH(c, "k_warm_perm");
    const int ge = (n * n + 255) / 256;
    const double couple = __builtin_popcount(c->eig_warm_hist) >= 4 ? kCouple : 0.0;
    // one refinement step in the form X = P (I + F) (see FProd): the products of small quantities in FP32,
    // E into T1, its largest entry into r32[0] (by k_refine_e), F <- F + E + F E
    auto refine_step = [&]() -> int {
      int s2;
      const FProd paf{N32, F32, Ap, F, AF, AF32, 0, 1, 0, 0, nullptr};  // A'F = D F + N F
      const FProd pff{F32, F32, nullptr, nullptr, FF, nullptr, 1, 0, 0, 0, nullptr};
      const FProd pfaf{F32, AF32, nullptr, nullptr, FAF, nullptr, 1, 0, 0, 0, nullptr};
      if ((s2 = fgemm(c, n, paf, nullptr)) || (s2 = fgemm(c, n, pff, &pfaf))) return s2;
      k_fassemble<<<ge, 256, 0, c->stream>>>(n, Ap, F, AF, FF, FAF, G, S, nrm, nnrm, S32, Gm32);
      PARO_LAUNCH(c, "k_fassemble");
      k_refine_lam<<<1, 1024, 0, c->stream>>>(n, G, S, nrm, nnrm, lam, cl, cst, ncl, r32, couple, S32, Gm32);
      PARO_LAUNCH(c, "k_refine_lam");
      k_refine_e<<<ge, 256, 0, c->stream>>>(n, G, S, lam, cl, T1, r32, E32);
      PARO_LAUNCH(c, "k_refine_e");
      const FProd pup{F32, E32, F, T1, Fn, Fn32, 0, 0, 0, 1, nullptr};  // F + E + F E
      if ((s2 = fgemm(c, n, pup, nullptr))) return s2;
      std::swap(F, Fn);
      std::swap(F32, Fn32);
      return PARO_OK;
    };
    auto read_emax = [&](float* e) -> int {
      void* h = nullptr;
      int s2 = d2h_async(c, "eig_warm_emax", r32, sizeof(float), &h);
      if (s2 || (s2 = pinned_wait(c, "eig_warm_emax"))) return s2;
      *e = *static_cast<const float*>(h);
      return PARO_OK;
    };
    // step 1 from the permutation, without products: G = I, S = A' (kept in Ap), F = E
    k_warm_s<<<nnrm, 256, 0, c->stream>>>(n, a, rk + n, G, Ap, nrm, nnrm, N32);
    PARO_LAUNCH(c, "k_warm_s");
    k_refine_lam<<<1, 1024, 0, c->stream>>>(n, G, Ap, nrm, nnrm, lam, cl, cst, ncl, nullptr, couple, N32, nullptr);
    PARO_LAUNCH(c, "k_refine_lam");
    k_refine_e<<<ge, 256, 0, c->stream>>>(n, G, Ap, lam, cl, F, nullptr, F32);
    PARO_LAUNCH(c, "k_refine_e");
    float emax = 1.f;
    if ((st = refine_step())) return st;
    // Well converged (the last warm start's correction below 1e-5; on the 64-atom cell near convergence the
    // second correction stays near 1e-6): the solve goes on without waiting, and the caller reads the
    // correction back with the Ritz values.
    const bool defer = emax_out && info_out && c->eig_warm_last < 1e-5f;
    if (defer) {
      void* h = nullptr;
      if ((st = d2h_async(c, "eig_warm_emax", r32, sizeof(float), &h))) return st;
      *emax_out = static_cast<const float*>(h);
      emax = 0.f;
    } else if ((st = read_emax(&emax))) {
      return st;
    }
    // a pair of close but separate eigenvalues converges more slowly: up to two more steps decide while the
    // correction still shrinks fast enough (measured on the 64-atom cell before convergence: the second
    // correction lies between 1e-4 and 1e-2 in most Rayleigh-Ritz steps; two more steps cost less than the
    // FP32 solve)
    if (emax >= 1e-4f && emax < 1e-1f && ((st = refine_step()) || (st = read_emax(&emax)))) return st;
    if (emax >= 1e-4f && emax < 1e-2f && ((st = refine_step()) || (st = read_emax(&emax)))) return st;
    prof_end(c, "eigh_warm", evw);
    if (defer || warm_outcome(c, emax)) {
      // finish in the same form: X' = I + F, T1 = A' X' = A' + A'F, S = X'^H A' X' inside the clusters,
      // Rayleigh-Ritz there on the columns of X', then X = P X'
      cudaEvent_t evf = prof_begin(c);
      const FProd pt{N32, F32, Ap, F, T1, nullptr, 0, 1, 1, 0, X};
      if ((st = fgemm(c, n, pt, nullptr))) return st;
      k_blockdiag_xhat<<<(int)((nn + 7) / 8), 256, 0, c->stream>>>(n, X, T1, cl, S);
      PARO_LAUNCH(c, "k_blockdiag_xhat");
      prof_end(c, "eigh_finish", evf);
      return eigh_finish_tail(c, n, a, X, S, cst, ncl, lam, w, v, perm, info, info_out, rk);
    }
    // not close enough: the FP32 solve (warm_outcome has set the calls to skip)
  }
  // the full Hermitian matrix (the input holds its lower triangle)
  k_herm_full_mixed<<<(int)((nn + 255) / 256), 256, 0, c->stream>>>(n, a, Af);
  PARO_LAUNCH(c, "k_herm_full");
  // 1. FP32 solve
  cudaEvent_t ev = prof_begin(c);
  const size_t sm1 = ((size_t)n * (n + 1) + 2 * (size_t)n) * sizeof(float2);
  PARO_CU(c, cudaFuncSetAttribute(k_tridiag_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  k_tridiag_cta<<<1, 1024, sm1, c->stream>>>(n, Af, U32, d32, e32, ph32, tau32, ecx32);
  PARO_LAUNCH(c, "k_tridiag_cta");
  prof_end(c, "k_tridiag_cta", ev);
  st = eigh_fp32_pieces(c, n, d32, e32, w32, U32, tau32, ph32, Z32, V32, info);
  if (st) return st;
  // 2. FP64 refinement (refine_steps steps), 3. Rayleigh-Ritz in the clusters
  ev = prof_begin(c);
  k_f2d<<<(int)((nn + 255) / 256), 256, 0, c->stream>>>((int)nn, V32, X);
  PARO_LAUNCH(c, "k_f2d");
  for (int it = 0; it < refine_steps; ++it) {
    if ((st = zgemm(c, n, X, true, X, G, false, part, true, nrm, true))) return st;          // G = X^H X
    if ((st = zgemm(c, n, Af, false, X, T1, false, part))) return st;                         // T1 = A X
    if ((st = zgemm(c, n, X, true, T1, S, false, part, true, nrm + nnrm, false))) return st;  // S = X^H A X
    cudaEvent_t ev2 = prof_begin(c);
    k_refine_lam<<<1, 1024, 0, c->stream>>>(n, G, S, nrm, nnrm, lam, cl, cst, ncl, nullptr, 0.0, nullptr,
                                            nullptr);
    PARO_LAUNCH(c, "k_refine_lam");
    prof_end(c, "k_refine_lam", ev2);
    ev2 = prof_begin(c);
    k_refine_e<<<(n * n + 255) / 256, 256, 0, c->stream>>>(n, G, S, lam, cl, T1, nullptr, nullptr);  // T1 = E
    PARO_LAUNCH(c, "k_refine_e");
    prof_end(c, "k_refine_e", ev2);
    if ((st = zgemm(c, n, X, false, T1, X, true, part))) return st;    // X += X E
  }
  prof_end(c, "eigh_refine", ev);
  return eigh_finish(c, n, a, Af, X, T1, S, part, cl, cst, ncl, lam, w, v, perm, info, refine_steps > 0, info_out);
}

// The end of the mixed solve from refined vectors X: T1 = A X, S = X^H A X (inside the clusters when they
// exist), Rayleigh-Ritz inside each cluster, eigenvalues sorted.
static int eigh_finish(Ctx* c, int n, const double2* a, const double2* Af, double2* X, double2* T1, double2* S,
                       double2* part, const int* cl, const int* cst, const int* ncl, double* lam, double* w,
                       double2* v, int* perm, int* info, bool clusters, const int** info_out) {
  const size_t nn = (size_t)n * n;
  int st;
  cudaEvent_t ev = prof_begin(c);
  if ((st = zgemm(c, n, Af, false, X, T1, false, part))) return st;    // T1 = A X
  if (clusters) {  // the clusters exist: S = X^H A X inside them only
    k_blockdiag_xhat<<<(int)((nn + 7) / 8), 256, 0, c->stream>>>(n, X, T1, cl, S);
    PARO_LAUNCH(c, "k_blockdiag_xhat");
  } else if ((st = zgemm(c, n, X, true, T1, S, false, part))) {
    return st;
  }
  prof_end(c, "eigh_finish", ev);
  return eigh_finish_tail(c, n, a, X, S, cst, ncl, lam, w, v, perm, info, info_out, nullptr);
}

// Rayleigh-Ritz inside the clusters on the columns of X, eigenvalues sorted (with rank, the rows put back in
// the original order: v = P X'); the cluster check is read back (or deferred via info_out).
static int eigh_finish_tail(Ctx* c, int n, const double2* a, double2* X, const double2* S, const int* cst,
                            const int* ncl, double* lam, double* w, double2* v, int* perm, int* info,
                            const int** info_out, const int* rank) {
  const size_t nn = (size_t)n * n;
  cudaEvent_t ev = prof_begin(c);
  const size_t sm3 = (size_t)2 * 64 * 65 * sizeof(double2);
  PARO_CU(c, cudaFuncSetAttribute(k_cluster_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  k_cluster_rr<<<n, 256, sm3, c->stream>>>(n, S, cst, ncl, X, lam, info);
  PARO_LAUNCH(c, "k_cluster_rr");
  k_eig_sort<<<(n + 127) / 128, 128, 0, c->stream>>>(n, lam, X, w, v, perm);
  PARO_LAUNCH(c, "k_eig_sort");
  k_eig_permute<<<(int)((nn + 255) / 256), 256, 0, c->stream>>>(n, lam, X, perm, rank, w, v);
  PARO_LAUNCH(c, "k_eig_permute");
  prof_end(c, "eigh_cluster_rr", ev);
  if (info_out) {  // the caller reads the cluster check later (eigh_mixed_check) without a wait here
    void* h = nullptr;
    int st = d2h_async(c, "eig_info", info, sizeof(int), &h);
    if (st) return st;
    *info_out = static_cast<const int*>(h);
    return PARO_OK;
  }
  int h = 0;
  PARO_CU(c, cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  return eigh_mixed_check(c, n, a, w, v, h);
}

int eigh_mixed_check(Ctx* c, int n, const double2* a, double* w, double2* v, int info) {
  if (info & 1) return fail(c, PARO_ERR_NOT_CONVERGED, "eigh (mixed): inverse iteration produced a zero vector");
  if (info & (4 | 8)) return eigh(c, n, a, w, v);  // a cluster the refinement cannot resolve: FP64 solver
  return PARO_OK;
}

}  // namespace paro
