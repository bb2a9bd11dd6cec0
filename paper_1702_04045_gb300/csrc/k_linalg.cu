// Dense complex linear algebra of the ParO projection step (Algorithm 1 step 4, Algorithm 2 step 4):
// Gram and Rayleigh-Ritz matrices (long-K "conj(A) B^T" GEMM, split over K with a fixed-order
// reduction), subspace rotations (short-K update GEMM), Cholesky orthonormalisation and the
// Hermitian eigensolver of the small Rayleigh-Ritz problem.
#include <cfloat>
#include <cmath>

#include "paro_ctx.h"

namespace paro {

template <typename A, typename B> struct Promote { using t = double; };
template <> struct Promote<float, float> { using t = float; };

template <typename TO, typename TI> __device__ __forceinline__ cplx<TO> cvt(cplx<TI> v) {
  return mk<TO>((TO)v.x, (TO)v.y);
}

// ------------------------------------------------------------------------------------------------
// C = conj(A) B^T, 32 x 32 output tile per CTA, K split over gridDim.z into fixed slices.
// part[z][m][n] receives the slice sums (complex double).
// ------------------------------------------------------------------------------------------------
template <typename TA, typename TB, typename ACC>
__global__ void __launch_bounds__(256) k_gemm_cn(int M, int N, int K, int kslice, const cplx<TA>* __restrict__ A,
                                                 int lda, const cplx<TB>* __restrict__ B, int ldb,
                                                 double2* __restrict__ part, int herm) {
  const int tm = blockIdx.y * 32, tn = blockIdx.x * 32;
  if (herm && tm > tn) return;
  const int k0 = blockIdx.z * kslice, k1 = min(K, k0 + kslice);
  __shared__ cplx<ACC> As[32][33], Bs[32][33];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  cplx<ACC> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = mk<ACC>(0, 0);
  for (int kk = k0; kk < k1; kk += 32) {
    for (int i = tid; i < 1024; i += 256) {
      const int r = i >> 5, kx = i & 31, gk = kk + kx;
      const int gm = tm + r, gn = tn + r;
      As[r][kx] = (gm < M && gk < k1) ? cconj(cvt<ACC, TA>(A[(size_t)gm * lda + gk])) : mk<ACC>(0, 0);
      Bs[r][kx] = (gn < N && gk < k1) ? cvt<ACC, TB>(B[(size_t)gn * ldb + gk]) : mk<ACC>(0, 0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kx = 0; kx < 32; ++kx) {
      const cplx<ACC> a0 = As[2 * ty][kx], a1 = As[2 * ty + 1][kx];
      const cplx<ACC> b0 = Bs[2 * tx][kx], b1 = Bs[2 * tx + 1][kx];
      acc[0][0] = cadd(acc[0][0], cmul(a0, b0));
      acc[0][1] = cadd(acc[0][1], cmul(a0, b1));
      acc[1][0] = cadd(acc[1][0], cmul(a1, b0));
      acc[1][1] = cadd(acc[1][1], cmul(a1, b1));
    }
    __syncthreads();
  }
  double2* pz = part + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = tm + 2 * ty + i, n = tn + 2 * tx + j;
      if (m < M && n < N) pz[(size_t)m * N + n] = make_double2((double)acc[i][j].x, (double)acc[i][j].y);
    }
}

__global__ void k_reduce_parts(int M, int N, int nz, const double2* __restrict__ part, double2* __restrict__ C,
                               int ldc, int herm) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int m = idx / N, n = idx - m * N;
  const bool mirror = herm && (m / 32) > (n / 32);
  const size_t off = mirror ? (size_t)n * N + m : (size_t)m * N + n;
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < nz; ++z) s = cadd(s, part[(size_t)z * M * N + off]);
  C[(size_t)m * ldc + n] = mirror ? cconj(s) : s;
}

template <typename TA, typename TB, typename ACC>
int gemm_cn(Ctx* c, int M, int N, int K, const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb, double2* C,
            int ldc, bool herm) {
  if (M <= 0 || N <= 0) return PARO_OK;
  const int tiles_m = (M + 31) / 32, tiles_n = (N + 31) / 32;
  const int tiles = herm ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
  int nz = (2 * 152 + tiles - 1) / tiles;
  const int maxz = (K + 255) / 256;
  if (nz > maxz) nz = maxz;
  if (nz < 1) nz = 1;
  const int kslice = ((K + nz - 1) / nz + 31) / 32 * 32;
  nz = (K + kslice - 1) / kslice;
  if (nz < 1) nz = 1;
  double2* part = static_cast<double2*>(ws_get(c, "gemm_parts", (size_t)nz * M * N * sizeof(double2)));
  if (!part) return PARO_ERR_CUDA;
  if (K == 0) {
    PARO_CU(c, cudaMemsetAsync(part, 0, (size_t)M * N * sizeof(double2), c->stream));
  } else {
    cudaEvent_t ev = prof_begin(c);
    k_gemm_cn<TA, TB, ACC><<<dim3(tiles_n, tiles_m, nz), 256, 0, c->stream>>>(M, N, K, kslice, A, lda, B, ldb, part,
                                                                              herm ? 1 : 0);
    PARO_LAUNCH(c, "k_gemm_cn");
    prof_end(c, sizeof(ACC) == 8 ? "k_gemm_cn<f64>" : "k_gemm_cn<f32>", ev);
  }
  k_reduce_parts<<<(M * N + 255) / 256, 256, 0, c->stream>>>(M, N, K == 0 ? 1 : nz, part, C, ldc, herm ? 1 : 0);
  PARO_LAUNCH(c, "k_reduce_parts");
  return PARO_OK;
}

// The same product with the K-slice partial sums in caller-provided memory of part_elems complex
// doubles (no allocation); every partial that k_reduce_parts reads is written first by k_gemm_cn.
template <typename TA, typename TB, typename ACC>
int gemm_cn_scratch(Ctx* c, int M, int N, int K, const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb,
                    double2* C, int ldc, double2* part, size_t part_elems) {
  if (M <= 0 || N <= 0) return PARO_OK;
  if (K <= 0) return fail(c, PARO_ERR_ARG, "gemm: K must be positive");
  const size_t slice = (size_t)M * N;
  if (part_elems < slice) return fail(c, PARO_ERR_ARG, "gemm: scratch smaller than one K slice");
  const int tiles = ((M + 31) / 32) * ((N + 31) / 32);
  int nz = (2 * 152 + tiles - 1) / tiles;
  const int maxz = (K + 255) / 256;
  if (nz > maxz) nz = maxz;
  if ((size_t)nz > part_elems / slice) nz = (int)(part_elems / slice);
  if (nz < 1) nz = 1;
  const int kslice = ((K + nz - 1) / nz + 31) / 32 * 32;
  nz = (K + kslice - 1) / kslice;
  k_gemm_cn<TA, TB, ACC><<<dim3((N + 31) / 32, (M + 31) / 32, nz), 256, 0, c->stream>>>(M, N, K, kslice, A, lda, B,
                                                                                      ldb, part, 0);
  PARO_LAUNCH(c, "k_gemm_cn");
  k_reduce_parts<<<(M * N + 255) / 256, 256, 0, c->stream>>>(M, N, nz, part, C, ldc, 0);
  PARO_LAUNCH(c, "k_reduce_parts");
  return PARO_OK;
}

template int gemm_cn_scratch<double, double, double>(Ctx*, int, int, int, const double2*, int, const double2*, int,
                                                     double2*, int, double2*, size_t);
template int gemm_cn_scratch<float, float, float>(Ctx*, int, int, int, const float2*, int, const float2*, int,
                                                  double2*, int, double2*, size_t);

// ------------------------------------------------------------------------------------------------
// Y = beta Y + W^T X (short K): 32 x 64 output tile per CTA, 256 threads with 4 x 2 outputs each.
// ------------------------------------------------------------------------------------------------
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) k_gemm_wx(int M, int N, int K, const double2* __restrict__ W, int ldw, int wt,
                                                 const double* __restrict__ s, const cplx<TX>* __restrict__ X,
                                                 int ldx, cplx<TY>* __restrict__ Y, int ldy, double beta) {
  const int tm = blockIdx.y * 32, tn = blockIdx.x * 64;
  __shared__ cplx<TY> Ws[16][32];
  __shared__ cplx<TY> Xs[16][64];
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  cplx<TY> acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = mk<TY>(0, 0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = tid; i < 16 * 32; i += 256) {
      const int kx = i >> 5, r = i & 31, gk = k0 + kx, gm = tm + r;
      double2 w = make_double2(0.0, 0.0);
      if (gk < K && gm < M) {
        w = wt ? W[(size_t)gm * ldw + gk] : W[(size_t)gk * ldw + gm];
        if (s) w = cscale(w, s[gk]);
      }
      Ws[kx][r] = mk<TY>((TY)w.x, (TY)w.y);
    }
    for (int i = tid; i < 16 * 64; i += 256) {
      const int kx = i >> 6, cc = i & 63, gk = k0 + kx, gn = tn + cc;
      Xs[kx][cc] = (gk < K && gn < N) ? cvt<TY, TX>(X[(size_t)gk * ldx + gn]) : mk<TY>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kx = 0; kx < 16; ++kx) {
      const cplx<TY> x0 = Xs[kx][tx], x1 = Xs[kx][tx + 32];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const cplx<TY> w = Ws[kx][ty * 4 + i];
        acc[i][0] = cadd(acc[i][0], cmul(w, x0));
        acc[i][1] = cadd(acc[i][1], cmul(w, x1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = tm + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = tn + tx + 32 * j;
      if (n >= N) continue;
      cplx<TY> v = acc[i][j];
      if (beta != 0.0) v = cadd(v, cscale(Y[(size_t)m * ldy + n], (TY)beta));
      Y[(size_t)m * ldy + n] = v;
    }
  }
}

template <typename TX, typename TY>
int gemm_wx(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s, const cplx<TX>* X,
            int ldx, cplx<TY>* Y, int ldy, double beta) {
  if (M <= 0 || N <= 0) return PARO_OK;
  cudaEvent_t ev = prof_begin(c);
  k_gemm_wx<TX, TY><<<dim3((N + 63) / 64, (M + 31) / 32), 256, 0, c->stream>>>(M, N, K, W, ldw, wt ? 1 : 0, s, X,
                                                                               ldx, Y, ldy, beta);
  PARO_LAUNCH(c, "k_gemm_wx");
  prof_end(c, sizeof(TY) == 8 ? "k_gemm_wx<f64>" : "k_gemm_wx<f32>", ev);
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Cholesky S = L L^H (left-looking, one CTA), then G = conj(L)^{-1} by forward substitution,
// one column of G per thread. info[0] = 0 or (1 + index of the first non-positive pivot).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_chol_inv(int n, const double2* __restrict__ S, double2* __restrict__ L,
                                                   double2* __restrict__ G, int* __restrict__ info) {
  __shared__ double red[32];
  __shared__ double s_diag;
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_bad = 0;
  for (int i = tid; i < n * n; i += nt) L[i] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int k = tid; k < j; k += nt) {
      const double2 l = L[(size_t)j * n + k];
      acc += l.x * l.x + l.y * l.y;
    }
    acc = block_sum(acc, red);
    if (tid == 0) {
      const double d = S[(size_t)j * n + j].x - acc;
      if (!(d > 0.0) || !isfinite(d)) {
        if (!s_bad) s_bad = j + 1;
        s_diag = 1.0;
      } else {
        s_diag = sqrt(d);
      }
      L[(size_t)j * n + j] = make_double2(s_diag, 0.0);
    }
    __syncthreads();
    const double ljj = s_diag;
    for (int i = j + 1 + tid; i < n; i += nt) {
      double2 v = S[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v = csub(v, cmul(L[(size_t)i * n + k], cconj(L[(size_t)j * n + k])));
      L[(size_t)i * n + j] = cscale(v, 1.0 / ljj);
    }
    __syncthreads();
  }
  // G = conj(L)^{-1}: column j solves conj(L) g = e_j.
  for (int j = tid; j < n; j += nt) {
    for (int i = 0; i < j; ++i) G[(size_t)i * n + j] = make_double2(0.0, 0.0);
    G[(size_t)j * n + j] = make_double2(1.0 / L[(size_t)j * n + j].x, 0.0);
    for (int i = j + 1; i < n; ++i) {
      double2 acc2 = make_double2(0.0, 0.0);
      for (int k = j; k < i; ++k) acc2 = cadd(acc2, cmul(cconj(L[(size_t)i * n + k]), G[(size_t)k * n + j]));
      G[(size_t)i * n + j] = cscale(acc2, -1.0 / L[(size_t)i * n + i].x);
    }
  }
  if (tid == 0) info[0] = s_bad;
}

int chol_inv(Ctx* c, int n, const double2* s, double2* g) {
  double2* L = static_cast<double2*>(ws_get(c, "chol_L", (size_t)n * n * sizeof(double2)));
  int* info = static_cast<int*>(ws_get(c, "chol_info", sizeof(int)));
  if (!L || !info) return PARO_ERR_CUDA;
  cudaEvent_t ev = prof_begin(c);
  k_chol_inv<<<1, 1024, 0, c->stream>>>(n, s, L, g, info);
  PARO_LAUNCH(c, "k_chol_inv");
  prof_end(c, "k_chol_inv", ev);
  int h = 0;
  PARO_CU(c, cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  if (h) return fail(c, PARO_ERR_BREAKDOWN, "Cholesky pivot <= 0 at column " + std::to_string(h - 1));
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Hermitian eigensolver, one CTA, FP64:
//  1. Householder reduction to tridiagonal form, A <- H_j A H_j with H_j = I - tau u u^H;
//  2. a diagonal unitary D makes the complex off-diagonals real and non-negative;
//  3. implicit-shift QL on the real tridiagonal matrix; thread 0 chases each bulge and records its
//     plane rotations, then every thread applies them to its own row of Z;
//  4. eigenvectors of A: Q D^H z, with Q = H_0 H_1 ..., sorted by ascending eigenvalue.
// work: n*n complex (A copy), n*n double (Z, column-major), info[0] = 0 or 1 if QL failed.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_eigh(int n, const double2* __restrict__ Ain, double2* __restrict__ A,
                                               double* __restrict__ Z, double* __restrict__ w,
                                               double2* __restrict__ V, double* __restrict__ dwork,
                                               int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* ph = reinterpret_cast<double2*>(smem_raw);  // n phases D_j
  double2* ecx = ph + n;                                // n complex off-diagonals
  double* d = reinterpret_cast<double*>(ecx + n);       // n
  double* e = d + n;                                    // n
  double* tau = e + n;                                  // n
  double* rs = tau + n;                                 // n rotation sines
  double* rcs = rs + n;                                 // n rotation cosines
  int* ri = reinterpret_cast<int*>(rcs + n);            // n rotation indices
  __shared__ double red[32];
  __shared__ double2 s_alpha;
  __shared__ double s_tau, s_K;
  __shared__ int s_cnt, s_go, s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  double2* p = reinterpret_cast<double2*>(dwork);     // n complex scratch (p, then w)

  // full Hermitian copy from the lower triangle
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    A[idx] = (i >= j) ? Ain[idx] : cconj(Ain[(size_t)j * n + i]);
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();

  // 1. tridiagonalisation
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1;             // length of x = A[j+1.., j]
    double nrm2 = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double2 x = A[(size_t)(j + 1 + i) * n + j];
      nrm2 += x.x * x.x + x.y * x.y;
    }
    nrm2 = block_sum(nrm2, red);
    if (tid == 0) {
      const double2 x0 = A[(size_t)(j + 1) * n + j];
      const double ax0 = hypot(x0.x, x0.y);
      const double nx = sqrt(nrm2);
      if (m == 1 || nx == 0.0 || nrm2 - ax0 * ax0 <= 0.0) {
        s_tau = 0.0;                     // nothing to annihilate
        s_alpha = x0;
      } else {
        const double2 phase = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
        s_alpha = make_double2(-phase.x * nx, -phase.y * nx);
        A[(size_t)(j + 1) * n + j] = csub(x0, s_alpha);  // u_0 = x_0 - alpha, u_i = x_i
        s_tau = 1.0 / (nrm2 + nx * ax0);                 // 2 / ||u||^2
      }
      tau[j] = s_tau;
      ecx[j] = s_alpha;
      d[j] = A[(size_t)j * n + j].x;
    }
    __syncthreads();
    const double t = s_tau;
    if (t != 0.0) {
      // u_i = A[(j+1+i)*n + j];  p = t * B u, B = A[j+1.., j+1..]; p_i = t * sum_k conj(B[k][i]) u_k (B Hermitian)
      for (int i = tid; i < m; i += nt) {
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < m; ++k)
          acc = cadd(acc, cmul(cconj(A[(size_t)(j + 1 + k) * n + (j + 1 + i)]), A[(size_t)(j + 1 + k) * n + j]));
        p[i] = cscale(acc, t);
      }
      __syncthreads();
      double kre = 0.0;  // u^H p is real
      for (int i = tid; i < m; i += nt) {
        const double2 ui = A[(size_t)(j + 1 + i) * n + j];
        const double2 pi = p[i];
        kre += ui.x * pi.x + ui.y * pi.y;
      }
      kre = block_sum(kre, red);
      if (tid == 0) s_K = 0.5 * t * kre;
      __syncthreads();
      for (int i = tid; i < m; i += nt) p[i] = csub(p[i], cscale(A[(size_t)(j + 1 + i) * n + j], s_K));  // w
      __syncthreads();
      // B -= u w^H + w u^H
      for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx / m, k = idx - i * m;
        const double2 ui = A[(size_t)(j + 1 + i) * n + j], uk = A[(size_t)(j + 1 + k) * n + j];
        const double2 wi = p[i], wk = p[k];
        double2& b = A[(size_t)(j + 1 + i) * n + (j + 1 + k)];
        b = csub(b, cadd(cmul(ui, cconj(wk)), cmul(wi, cconj(uk))));
      }
      __syncthreads();
    }
  }
  if (tid == 0) d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)].x;
  __syncthreads();

  // 2. phases: D_0 = 1, D_{j+1} = D_j conj(e_j)/|e_j|; real off-diagonals |e_j|
  if (tid == 0) {
    ph[0] = make_double2(1.0, 0.0);
    for (int j = 0; j + 1 < n; ++j) {
      const double a = hypot(ecx[j].x, ecx[j].y);
      e[j] = a;
      ph[j + 1] = a > 0.0 ? cmul(ph[j], make_double2(ecx[j].x / a, -ecx[j].y / a)) : ph[j];
    }
    e[n - 1] = 0.0;
  }
  for (int idx = tid; idx < n * n; idx += nt) Z[idx] = 0.0;
  __syncthreads();
  for (int k = tid; k < n; k += nt) Z[(size_t)k * n + k] = 1.0;  // Z column-major: Z[col*n + row]
  __syncthreads();

  // 3. implicit QL; rotation (i, s, c) acts on columns i, i+1 of Z
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      if (tid == 0) {
        int m = l;
        for (; m < n - 1; ++m) {
          const double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= DBL_EPSILON * dd) break;
        }
        if (m == l) {
          s_go = 0;
        } else if (iter >= 60) {
          s_bad = 1;
          s_go = 0;
        } else {
          ++iter;
          double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
          double r = hypot(g, 1.0);
          g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
          double s = 1.0, cs = 1.0, pp = 0.0;
          int cnt = 0;
          bool early = false;
          for (int i = m - 1; i >= l; --i) {
            const double f = s * e[i], b = cs * e[i];
            r = hypot(f, g);
            e[i + 1] = r;
            if (r == 0.0) {
              d[i + 1] -= pp;
              e[m] = 0.0;
              early = true;
              break;
            }
            s = f / r;
            cs = g / r;
            g = d[i + 1] - pp;
            r = (d[i] - g) * s + 2.0 * cs * b;
            pp = s * r;
            d[i + 1] = g + pp;
            g = cs * r - b;
            ri[cnt] = i;
            rs[cnt] = s;
            rcs[cnt] = cs;
            ++cnt;
          }
          if (!early) {
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
          }
          s_cnt = cnt;
          s_go = 1;
        }
      }
      __syncthreads();
      if (!s_go) break;
      const int cnt = s_cnt;
      for (int k = tid; k < n; k += nt) {
        for (int t = 0; t < cnt; ++t) {
          const int i = ri[t];
          const double s = rs[t], cs = rcs[t];
          const double zi = Z[(size_t)i * n + k], zi1 = Z[(size_t)(i + 1) * n + k];
          Z[(size_t)(i + 1) * n + k] = s * zi + cs * zi1;
          Z[(size_t)i * n + k] = cs * zi - s * zi1;
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();

  // 4. sort and back-transform: column r(k) of V = Q D^H z_k
  for (int k = tid; k < n; k += nt) {
    int r = 0;
    const double dk = d[k];
    for (int j = 0; j < n; ++j) r += (d[j] < dk) || (d[j] == dk && j < k);
    w[r] = dk;
    for (int i = 0; i < n; ++i) V[(size_t)i * n + r] = cscale(cconj(ph[i]), Z[(size_t)k * n + i]);
  }
  __syncthreads();
  for (int j = n - 2; j >= 0; --j) {
    const double t = tau[j];
    if (t == 0.0) continue;
    const int m = n - j - 1;
    for (int col = tid; col < n; col += nt) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < m; ++i) s = cadd(s, cmul(cconj(A[(size_t)(j + 1 + i) * n + j]), V[(size_t)(j + 1 + i) * n + col]));
      s = cscale(s, t);
      for (int i = 0; i < m; ++i) {
        double2& v = V[(size_t)(j + 1 + i) * n + col];
        v = csub(v, cmul(A[(size_t)(j + 1 + i) * n + j], s));
      }
    }
    __syncthreads();
  }
  if (tid == 0) info[0] = s_bad;
}

int eigh(Ctx* c, int n, const double2* a, double* w, double2* v) {
  if (n < 1 || n > 4096) return fail(c, PARO_ERR_ARG, "eigh: n out of range");
  double2* A = static_cast<double2*>(ws_get(c, "eigh_A", (size_t)n * n * sizeof(double2)));
  double* Z = static_cast<double*>(ws_get(c, "eigh_Z", (size_t)n * n * sizeof(double)));
  double* dw = static_cast<double*>(ws_get(c, "eigh_p", (size_t)n * sizeof(double2)));
  int* info = static_cast<int*>(ws_get(c, "eigh_info", sizeof(int)));
  if (!A || !Z || !dw || !info) return PARO_ERR_CUDA;
  const size_t smem = (size_t)n * (5 * sizeof(double) + 2 * sizeof(double2) + sizeof(int));
  if (smem > 227 * 1024) return fail(c, PARO_ERR_ARG, "eigh: n too large for shared memory");
  PARO_CU(c, cudaFuncSetAttribute(k_eigh, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int threads = ((n + 31) / 32) * 32;
  if (threads < 256) threads = 256;
  if (threads > 1024) threads = 1024;
  cudaEvent_t ev = prof_begin(c);
  k_eigh<<<1, threads, smem, c->stream>>>(n, a, A, Z, w, v, dw, info);
  PARO_LAUNCH(c, "k_eigh");
  prof_end(c, "k_eigh", ev);
  int h = 0;
  PARO_CU(c, cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  if (h) return fail(c, PARO_ERR_NOT_CONVERGED, "eigh: QL iteration limit reached");
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// per-band reductions
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_band_norm2(int npw, const cplx<T>* __restrict__ x, int ldx, double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const cplx<T>* xb = x + (size_t)b * ldx;
  double acc = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double re = xb[g].x, im = xb[g].y;
    acc += re * re + im * im;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[b] = acc;
}

template <typename T>
int band_norms(Ctx* c, int nb, int npw, const cplx<T>* x, int ldx, double* out_dev) {
  k_band_norm2<T><<<nb, 256, 0, c->stream>>>(npw, x, ldx, out_dev);
  PARO_LAUNCH(c, "k_band_norm2");
  return PARO_OK;
}

__global__ void k_resid(int npw, const double2* __restrict__ psi, const double2* __restrict__ hpsi,
                        const double* __restrict__ eps, double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const double e = eps[b];
  double acc = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 p = psi[(size_t)b * npw + g], h = hpsi[(size_t)b * npw + g];
    const double re = h.x - e * p.x, im = h.y - e * p.y;
    acc += re * re + im * im;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[b] = sqrt(acc);
}

int residual_norms(Ctx* c, int nb, int npw, const double2* psi, const double2* hpsi, const double* eps_dev,
                   double* out_dev) {
  k_resid<<<nb, 256, 0, c->stream>>>(npw, psi, hpsi, eps_dev, out_dev);
  PARO_LAUNCH(c, "k_resid");
  return PARO_OK;
}

template <typename TS, typename TD>
__global__ void k_convert(size_t n, const cplx<TS>* __restrict__ s, cplx<TD>* __restrict__ d) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = mk<TD>((TD)s[i].x, (TD)s[i].y);
}

template <typename TS, typename TD>
int convert(Ctx* c, size_t n, const cplx<TS>* src, cplx<TD>* dst) {
  if (n == 0) return PARO_OK;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_convert<TS, TD><<<blocks, 256, 0, c->stream>>>(n, src, dst);
  PARO_LAUNCH(c, "k_convert");
  return PARO_OK;
}

// instantiations
template int gemm_cn<double, double, double>(Ctx*, int, int, int, const double2*, int, const double2*, int, double2*,
                                             int, bool);
template int gemm_cn<float, float, float>(Ctx*, int, int, int, const float2*, int, const float2*, int, double2*, int,
                                          bool);
template int gemm_cn<float, float, double>(Ctx*, int, int, int, const float2*, int, const float2*, int, double2*,
                                           int, bool);
template int gemm_cn<double, float, double>(Ctx*, int, int, int, const double2*, int, const float2*, int, double2*,
                                            int, bool);
template int gemm_wx<double, double>(Ctx*, int, int, int, const double2*, int, bool, const double*, const double2*,
                                     int, double2*, int, double);
template int gemm_wx<float, float>(Ctx*, int, int, int, const double2*, int, bool, const double*, const float2*, int,
                                   float2*, int, double);
template int gemm_wx<float, double>(Ctx*, int, int, int, const double2*, int, bool, const double*, const float2*,
                                    int, double2*, int, double);
template int band_norms<double>(Ctx*, int, int, const double2*, int, double*);
template int band_norms<float>(Ctx*, int, int, const float2*, int, double*);
template int convert<double, float>(Ctx*, size_t, const double2*, float2*);
template int convert<float, double>(Ctx*, size_t, const float2*, double2*);

}  // namespace paro
