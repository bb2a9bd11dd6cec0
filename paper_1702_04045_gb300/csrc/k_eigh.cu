// Hermitian eigensolver of the Rayleigh-Ritz step (Algorithm 1 step 4; Algorithm 2 step 4), FP64.
// GB300 runs FP64 at about 2 FMA per clock per SM, so every O(n^3) part is spread over many SMs:
//
//  1. k_tridiag_cluster (one thread-block cluster of 16 or 8 CTAs, the matrix in their distributed shared
//     memory) or, when it does not fit, k_tridiag (cooperative, many CTAs, grid barriers): Householder
//     reduction A <- H_j A H_j, H_j = I - tau u u^H, to a Hermitian tridiagonal matrix. A diagonal
//     unitary D (D_0 = 1, D_{j+1} = D_j conj(e_j)/|e_j|) turns the complex off-diagonals e_j into |e_j|:
//     a real symmetric tridiagonal T'.
//  2. k_bisect (warp per eigenvalue): the k-th eigenvalue of T' by multisection on the Sturm count
//     (the number of negative pivots of the LDL^T factorisation of T' - x), 32 points per step.
//  3. k_invit_solve / k_invit_mgs: eigenvectors of T' by inverse iteration, one thread per eigenvalue
//     with its LU factorisation of T' - lambda (partial pivoting) and its vector in shared memory; after
//     each of three solves the vectors of a cluster (eigenvalues closer than 1e-3 ||T'||_1) are
//     orthogonalised in eigenvalue order by one warp (the standard remedy for close eigenvalues, as in
//     LAPACK's xSTEIN).
//  4. k_backtransform (warp per column, many CTAs): eigenvectors of A = Q D^H z, Q = H_0 H_1 ...
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "paro_ctx.h"

namespace cg = cooperative_groups;

namespace paro {

__global__ void k_herm_full(int n, const double2* __restrict__ Ain, double2* __restrict__ A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  A[idx] = (i >= j) ? Ain[idx] : cconj(Ain[(size_t)j * n + i]);
}

// -------------------------------------------------------------------------------------------------
// 1. tridiagonalisation. A: n x n full Hermitian work copy; u_j ends up below the diagonal of column
// j. ub, pb: n complex of scratch; sc: scalars; bar: grid barrier; err: barrier time-out flag.
// -------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tridiag(int n, double2* __restrict__ A, double* __restrict__ d,
                                                 double* __restrict__ e, double2* __restrict__ ph,
                                                 double* __restrict__ tau, double2* __restrict__ ecx,
                                                 double2* __restrict__ ub, double2* __restrict__ pb,
                                                 double* __restrict__ sc, unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* us = reinterpret_cast<double2*>(smem_raw);  // u
  double2* ws = us + n;                                 // w
  __shared__ double red[32];
  __shared__ double s_K;
  const int tid = threadIdx.x, lane = tid & 31;
  const int gwarp = blockIdx.x * (blockDim.x >> 5) + (tid >> 5), nwarp = gridDim.x * (blockDim.x >> 5);
  const int gth = blockIdx.x * blockDim.x + tid, nth = gridDim.x * blockDim.x;
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1;
    if (blockIdx.x == 0) {  // the reflector of column j
      double nrm2 = 0.0;
      for (int i = tid; i < m; i += blockDim.x) {
        const double2 x = __ldcg(&A[(size_t)(j + 1 + i) * n + j]);
        us[i] = x;
        nrm2 += x.x * x.x + x.y * x.y;
      }
      nrm2 = block_sum(nrm2, red);
      if (tid == 0) {
        const double2 x0 = us[0];
        const double ax0 = hypot(x0.x, x0.y);
        const double nx = sqrt(nrm2);
        double2 alpha = x0;
        double t = 0.0;
        if (m > 1 && nx > 0.0 && nrm2 - ax0 * ax0 > 0.0) {
          const double2 phs = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
          alpha = make_double2(-phs.x * nx, -phs.y * nx);
          us[0] = csub(x0, alpha);  // u = x - alpha e_1
          __stcg(&A[(size_t)(j + 1) * n + j], us[0]);
          t = 1.0 / (nrm2 + nx * ax0);  // 2 / ||u||^2
        }
        sc[j & 1] = t;  // by parity: a CTA still reading step j's t while block 0 starts j + 1
        tau[j] = t;
        ecx[j] = alpha;
        d[j] = __ldcg(&A[(size_t)j * n + j]).x;
      }
      __syncthreads();
      for (int i = tid; i < m; i += blockDim.x) __stcg(&ub[i], us[i]);
    }
    if (!grid_barrier(bar, err)) return;
    const double t = __ldcg(&sc[j & 1]);
    if (t == 0.0) continue;
    for (int i = tid; i < m; i += blockDim.x) us[i] = __ldcg(&ub[i]);
    __syncthreads();
    // p_i = t sum_k B[i][k] u_k, B = A[j+1.., j+1..]: one warp per row
    for (int i = gwarp; i < m; i += nwarp) {
      const double2* row = A + (size_t)(j + 1 + i) * n + (j + 1);
      double2 acc = make_double2(0.0, 0.0);
      for (int k = lane; k < m; k += 32) {
        const double2 b = __ldcg(&row[k]), u = us[k];
        acc.x = fma(b.x, u.x, fma(-b.y, u.y, acc.x));
        acc.y = fma(b.x, u.y, fma(b.y, u.x, acc.y));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) __stcg(&pb[i], cscale(acc, t));
    }
    if (!grid_barrier(bar, err)) return;
    double kre = 0.0;  // u^H p is real; every CTA forms it
    for (int i = tid; i < m; i += blockDim.x) {
      const double2 p = __ldcg(&pb[i]);
      ws[i] = p;
      kre += us[i].x * p.x + us[i].y * p.y;
    }
    kre = block_sum(kre, red);
    if (tid == 0) s_K = 0.5 * t * kre;
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) ws[i] = csub(ws[i], cscale(us[i], s_K));  // w = p - K u
    __syncthreads();
    for (size_t idx = gth; idx < (size_t)m * m; idx += nth) {  // B -= u w^H + w u^H
      const int i = (int)(idx / m), k = (int)(idx - (size_t)i * m);
      double2* bp = &A[(size_t)(j + 1 + i) * n + (j + 1 + k)];
      const double2 ui = us[i], wi = ws[i], uk = us[k], wk = ws[k];
      double2 b = __ldcg(bp);
      b.x -= ui.x * wk.x + ui.y * wk.y + wi.x * uk.x + wi.y * uk.y;
      b.y -= ui.y * wk.x - ui.x * wk.y + wi.y * uk.x - wi.x * uk.y;
      __stcg(bp, b);
    }
    if (!grid_barrier(bar, err)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    d[n - 1] = __ldcg(&A[(size_t)(n - 1) * n + (n - 1)]).x;
    ph[0] = make_double2(1.0, 0.0);
    for (int j = 0; j + 1 < n; ++j) {
      const double a = hypot(ecx[j].x, ecx[j].y);
      e[j] = a;
      ph[j + 1] = a > 0.0 ? cmul(ph[j], make_double2(ecx[j].x / a, -ecx[j].y / a)) : ph[j];
    }
    e[n - 1] = 0.0;
  }
}

// -------------------------------------------------------------------------------------------------
// 1'. the same reduction on one thread-block cluster of C CTAs, for matrices that fit in the cluster's
// shared memory: row g of the full Hermitian matrix lives in CTA g mod C (local row g / C), so the
// active rows stay spread evenly as the matrix shrinks. Step j: the owner of row j forms u_j from it
// (column j below the diagonal is the conjugate of row j right of it); cluster barrier; every CTA reads
// u_j from the owner's shared memory and forms p_i = tau sum_k B_ik u_k for its rows; cluster barrier;
// every CTA gathers all of p, forms w = p - (tau/2)(u^H p) u in the same order, and updates its rows
// B -= u w^H + w u^H. u_j is written to U[j][0..m) for the back-transformation. Buffers shared with
// other CTAs alternate with the step parity; a barrier separates every write from the reads of the
// step before that used the same buffer.
// -------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tridiag_cluster(int n, const double2* __restrict__ a,
                                                          double2* __restrict__ U, double* __restrict__ d,
                                                          double* __restrict__ e, double2* __restrict__ ph,
                                                          double* __restrict__ tau, double2* __restrict__ ecx) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int R = (n + C - 1) / C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* rows = reinterpret_cast<double2*>(smem_raw);  // R x n
  double2* ubuf = rows + (size_t)R * n;                  // 2 x n: u_j of the steps this CTA owns
  double2* pl = ubuf + 2 * n;                            // 2 x n: p_i of this CTA's rows, i = g - j - 1
  double2* ul = pl + 2 * n;                              // u_j (local copy)
  double2* wl = ul + n;                                  // p, then w
  double* tb = reinterpret_cast<double*>(wl + n);        // 2: tau_j of owned steps
  __shared__ double red[32];
  __shared__ double s_K;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (size_t idx = tid; idx < (size_t)R * n; idx += blockDim.x) {
    const int r = (int)(idx / n), k = (int)(idx - (size_t)r * n), g = q + C * r;
    rows[idx] = g >= n ? make_double2(0.0, 0.0) : (g >= k ? a[(size_t)g * n + k] : cconj(a[(size_t)k * n + g]));
  }
  __syncthreads();
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1, par = j & 1, owner = j % C;
    double2* ub = ubuf + par * n;
    if (q == owner) {
      const double2* rj = rows + (size_t)(j / C) * n;
      double nrm2 = 0.0;
      for (int i = tid; i < m; i += blockDim.x) {
        const double2 x = cconj(rj[j + 1 + i]);
        ub[i] = x;
        nrm2 += x.x * x.x + x.y * x.y;
      }
      nrm2 = block_sum(nrm2, red);
      if (tid == 0) {
        const double2 x0 = ub[0];
        const double ax0 = hypot(x0.x, x0.y);
        const double nx = sqrt(nrm2);
        double2 alpha = x0;
        double t = 0.0;
        if (m > 1 && nx > 0.0 && nrm2 - ax0 * ax0 > 0.0) {
          const double2 phs = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
          alpha = make_double2(-phs.x * nx, -phs.y * nx);
          ub[0] = csub(x0, alpha);  // u = x - alpha e_1
          t = 1.0 / (nrm2 + nx * ax0);  // 2 / ||u||^2
        }
        tb[par] = t;
        tau[j] = t;
        ecx[j] = alpha;
        d[j] = rj[j].x;
      }
      __syncthreads();
      for (int i = tid; i < m; i += blockDim.x) U[(size_t)j * n + i] = ub[i];
    }
    cl.sync();
    const double t = *cl.map_shared_rank(tb + par, owner);
    if (t == 0.0) continue;  // the same t in every CTA: all skip the step together
    const double2* uo = cl.map_shared_rank(ub, owner);
    for (int i = tid; i < m; i += blockDim.x) ul[i] = uo[i];
    __syncthreads();
    const int r0 = (j + 1 > q) ? (j + 1 - q + C - 1) / C : 0;  // first local row with g > j
    for (int r = r0 + warp; r < R; r += nwarp) {
      const int g = q + C * r;
      if (g >= n) break;
      const double2* row = rows + (size_t)r * n + (j + 1);
      double2 acc = make_double2(0.0, 0.0);
      for (int k = lane; k < m; k += 32) {
        const double2 b = row[k], u = ul[k];
        acc.x = fma(b.x, u.x, fma(-b.y, u.y, acc.x));
        acc.y = fma(b.x, u.y, fma(b.y, u.x, acc.y));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) pl[par * n + (g - j - 1)] = cscale(acc, t);
    }
    cl.sync();
    double kre = 0.0;  // u^H p is real
    for (int i = tid; i < m; i += blockDim.x) {
      const double2 p = *cl.map_shared_rank(pl + par * n + i, (j + 1 + i) % C);
      wl[i] = p;
      kre += ul[i].x * p.x + ul[i].y * p.y;
    }
    kre = block_sum(kre, red);
    if (tid == 0) s_K = 0.5 * t * kre;
    __syncthreads();
    const double K = s_K;
    for (int i = tid; i < m; i += blockDim.x) wl[i] = csub(wl[i], cscale(ul[i], K));  // w = p - K u
    __syncthreads();
    for (int r = r0 + warp; r < R; r += nwarp) {  // B -= u w^H + w u^H on this CTA's rows
      const int g = q + C * r;
      if (g >= n) break;
      const int i = g - j - 1;
      const double2 ui = ul[i], wi = wl[i];
      double2* row = rows + (size_t)r * n + (j + 1);
      for (int k = lane; k < m; k += 32) {
        const double2 uk = ul[k], wk = wl[k];
        double2 b = row[k];
        b.x -= ui.x * wk.x + ui.y * wk.y + wi.x * uk.x + wi.y * uk.y;
        b.y -= ui.y * wk.x - ui.x * wk.y + wi.y * uk.x - wi.x * uk.y;
        row[k] = b;
      }
    }
    __syncthreads();
  }
  if (q == (n - 1) % C && tid == 0) d[n - 1] = rows[(size_t)((n - 1) / C) * n + (n - 1)].x;
  __threadfence();
  cl.sync();  // no CTA leaves while another may still read its shared memory; d and ecx complete
  if (q == 0 && tid == 0) {
    ph[0] = make_double2(1.0, 0.0);
    for (int j = 0; j + 1 < n; ++j) {
      const double v = hypot(ecx[j].x, ecx[j].y);
      e[j] = v;
      ph[j + 1] = v > 0.0 ? cmul(ph[j], make_double2(ecx[j].x / v, -ecx[j].y / v)) : ph[j];
    }
    e[n - 1] = 0.0;
  }
}

// -------------------------------------------------------------------------------------------------
// 2. multisection: w[k] = k-th smallest eigenvalue of T' (d, e); one warp per eigenvalue. R = double,
// or float for the first stage of the mixed-precision solver (refined afterwards in FP64).
// -------------------------------------------------------------------------------------------------
template <typename R> struct RealLimits;
template <> struct RealLimits<double> {
  static __device__ __forceinline__ double eps() { return DBL_EPSILON; }
  static __device__ __forceinline__ double tiny() { return DBL_MIN; }
  static __device__ __forceinline__ double huge() { return 1e300; }
};
template <> struct RealLimits<float> {
  static __device__ __forceinline__ float eps() { return FLT_EPSILON; }
  static __device__ __forceinline__ float tiny() { return FLT_MIN; }
  static __device__ __forceinline__ float huge() { return 1e30f; }
};

template <typename R>
__device__ __forceinline__ int sturm_count(int n, const R* d, const R* e2, R x, R pivmin) {
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < (R)0;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < (R)0;
  }
  return c;
}

template <typename R>
__global__ void __launch_bounds__(128) k_bisect(int n, const R* __restrict__ dg, const R* __restrict__ eg,
                                                R* __restrict__ w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* d = reinterpret_cast<R*>(smem_raw);
  R* e2 = d + n;
  __shared__ R s_lo, s_hi, s_pivmin;
  using L = RealLimits<R>;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = dg[i];
    e2[i] = eg[i] * eg[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R lo = L::huge(), hi = -L::huge(), emax = 0;
    for (int i = 0; i < n; ++i) {
      const R r = (i > 0 ? fabs(eg[i - 1]) : (R)0) + (i + 1 < n ? fabs(eg[i]) : (R)0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      emax = fmax(emax, e2[i]);
    }
    const R tn = fmax(fabs(lo), fabs(hi));
    s_lo = lo - (R)2 * L::eps() * tn * n - L::tiny();
    s_hi = hi + (R)2 * L::eps() * tn * n + L::tiny();
    s_pivmin = L::tiny() * fmax((R)1, emax);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= n) return;
  R lo = s_lo, hi = s_hi;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= (R)2 * L::eps() * fmax(fabs(lo), fabs(hi)) + s_pivmin) break;
    const R x = lo + (hi - lo) * (R)(lane + 1) / (R)33;
    const int cnt = sturm_count<R>(n, d, e2, x, s_pivmin);
    const unsigned above = __ballot_sync(0xffffffffu, cnt > k);
    const int l = above ? __ffs(above) - 1 : 32;  // first point with more than k eigenvalues below it
    const R xl = __shfl_sync(0xffffffffu, x, l < 32 ? l : 31);
    const R xm = __shfl_sync(0xffffffffu, x, l > 0 ? l - 1 : 0);
    const R nlo = l == 0 ? lo : xm;
    const R nhi = l == 32 ? hi : xl;
    if (!(nhi - nlo < hi - lo)) break;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) w[k] = (R)0.5 * (lo + hi);
}

// -------------------------------------------------------------------------------------------------
// 3. inverse iteration. Shifts: eigenvalues closer than ortol = 1e-3 ||T'||_1 form a cluster, and shifts
// inside a cluster are kept at least 10 eps |lambda| + eps ||T'||_1 apart (k_invit_prep, one thread).
// k_invit_solve: one thread per eigenvalue, EPB per CTA, the LU factorisation of T' - lambda_j (partial
// pivoting) and the vector in shared memory ([row][thread], conflict free); solves (T' - lambda_j) z = z
// from the stored vector (or a fixed start vector) and writes it back. k_invit_mgs: the vectors of each
// cluster are orthonormalised in eigenvalue order by one warp (the standard remedy for close eigenvalues,
// as in LAPACK's xSTEIN). Three rounds of solve + orthonormalisation. Z: column j = vector j (n x n).
// -------------------------------------------------------------------------------------------------
template <typename R>
__global__ void k_invit_prep(int n, const R* __restrict__ d, const R* __restrict__ e, const R* __restrict__ w,
                             R* __restrict__ lam, int* __restrict__ cstart, int* __restrict__ nclu,
                             R* __restrict__ tiny_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  using L = RealLimits<R>;
  const R eps = L::eps();
  R t1 = 0;
  for (int i = 0; i < n; ++i)
    t1 = fmax(t1, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : (R)0) + (i + 1 < n ? fabs(e[i]) : (R)0));
  t1 = fmax(t1, L::tiny());
  const R ortol = (R)1e-3 * t1, tiny = eps * t1;
  int nc = 0;
  for (int j = 0; j < n; ++j) {
    R l = w[j];
    if (j == 0 || w[j] - w[j - 1] > ortol) {
      cstart[nc++] = j;
    } else if (l - lam[j - 1] < (R)10 * eps * fabs(l) + tiny) {
      l = lam[j - 1] + (R)10 * eps * fabs(l) + tiny;
    }
    lam[j] = l;
  }
  cstart[nc] = n;
  *nclu = nc;
  *tiny_out = tiny;
}

// The factors depend only on lambda_j: the first round stores them in fac (4 n x n values, [i][j]) and
// sw (n x n), later rounds read them back instead of factorising again.
template <typename R>
__global__ void k_invit_solve(int n, const R* __restrict__ d, const R* __restrict__ e, const R* __restrict__ lam,
                              const R* __restrict__ tinyp, R* __restrict__ Z, int first, R* __restrict__ fac,
                              unsigned char* __restrict__ swg, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int E = blockDim.x, t = threadIdx.x, j = blockIdx.x * E + t;
  R* R0 = reinterpret_cast<R*>(smem_raw);  // 1 / (guarded pivot)
  R* U1 = R0 + (size_t)n * E;
  R* U2 = U1 + (size_t)n * E;
  R* Lm = U2 + (size_t)n * E;
  R* z = Lm + (size_t)n * E;
  unsigned char* SW = reinterpret_cast<unsigned char*>(z + (size_t)n * E);
  if (j >= n) return;  // no barriers below
  const size_t nn = (size_t)n * n;
  if (!first) {
#pragma unroll 8
    for (int i = 0; i < n; ++i) {  // independent loads: unrolled so that many are in flight
      const size_t o = (size_t)i * E + t, g = (size_t)i * n + j;
      R0[o] = fac[g]; U1[o] = fac[nn + g]; U2[o] = fac[2 * nn + g]; Lm[o] = fac[3 * nn + g]; SW[o] = swg[g];
    }
  } else {
  const R tiny = *tinyp, l = lam[j];
  R p = d[0] - l, q = n > 1 ? e[0] : (R)0, r = 0;
  for (int i = 0; i + 1 < n; ++i) {  // LU of T' - l with partial pivoting, row i at [i * E + t]
    const R b = e[i];
    const R a1 = d[i + 1] - l, c1 = (i + 2 < n) ? e[i + 1] : (R)0;
    R u0, u1, u2, mlt;
    unsigned char sw;
    if (fabs(p) >= fabs(b)) {
      mlt = (p != (R)0) ? b / p : (R)0;
      u0 = p; u1 = q; u2 = r; sw = 0;
      p = a1 - mlt * q;
      q = c1 - mlt * r;
    } else {
      mlt = p / b;
      u0 = b; u1 = a1; u2 = c1; sw = 1;
      p = q - mlt * a1;
      q = r - mlt * c1;
    }
    r = 0;
    if (fabs(u0) < tiny) u0 = u0 < (R)0 ? -tiny : tiny;
    const size_t o = (size_t)i * E + t;
    R0[o] = (R)1 / u0; U1[o] = u1; U2[o] = u2; Lm[o] = mlt; SW[o] = sw;
  }
  if (fabs(p) < tiny) p = p < (R)0 ? -tiny : tiny;
  {
    const size_t o = (size_t)(n - 1) * E + t;
    R0[o] = (R)1 / p; U1[o] = 0; U2[o] = 0; Lm[o] = 0; SW[o] = 0;
  }
  for (int i = 0; i < n; ++i) {
    const size_t o = (size_t)i * E + t, g = (size_t)i * n + j;
    fac[g] = R0[o]; fac[nn + g] = U1[o]; fac[2 * nn + g] = U2[o]; fac[3 * nn + g] = Lm[o]; swg[g] = SW[o];
  }
  }
#pragma unroll 8
  for (int i = 0; i < n; ++i)
    z[(size_t)i * E + t] = first ? (R)(((i * 7919 + j * 104729) % 1999) + 1) / (R)1999 - (R)0.5 : Z[(size_t)i * n + j];
  for (int i = 0; i + 1 < n; ++i) {  // forward: row interchanges and multipliers
    const size_t o = (size_t)i * E + t;
    R zi = z[o], zi1 = z[o + E];
    if (SW[o]) { const R tmp = zi; zi = zi1; zi1 = tmp; }
    z[o] = zi;
    z[o + E] = zi1 - Lm[o] * zi;
  }
  R nrm = 0;
  for (int i = n - 1; i >= 0; --i) {  // back substitution with U (bandwidth 3)
    const size_t o = (size_t)i * E + t;
    R sv = z[o];
    if (i + 1 < n) sv -= U1[o] * z[o + E];
    if (i + 2 < n) sv -= U2[o] * z[o + 2 * E];
    sv *= R0[o];
    z[o] = sv;
    nrm += sv * sv;
  }
  // normalised here (k_invit_mgs orthogonalises and normalises again inside clusters of two or more)
  if (!(nrm > (R)0) || !isfinite(nrm)) {
    atomicExch(info, 1);
    nrm = 1;
  }
  const R inv = (R)1 / sqrt(nrm);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + j] = z[(size_t)i * E + t] * inv;
}

template <typename R>
__global__ void k_invit_mgs(int n, R* __restrict__ Z, const int* __restrict__ cstart, const int* __restrict__ nclu,
                            int* __restrict__ info) {
  const int lane = threadIdx.x & 31;
  const int cl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (cl >= *nclu) return;
  const int c0 = cstart[cl], c1 = cstart[cl + 1];
  if (c1 - c0 < 2) return;  // a single vector: k_invit_solve has normalised it
  for (int j = c0; j < c1; ++j) {
    for (int q = c0; q < j; ++q) {
      R s = 0;
      for (int i = lane; i < n; i += 32) s += Z[(size_t)i * n + j] * Z[(size_t)i * n + q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      for (int i = lane; i < n; i += 32) Z[(size_t)i * n + j] -= s * Z[(size_t)i * n + q];
      __syncwarp();
    }
    R nrm = 0;
    for (int i = lane; i < n; i += 32) nrm += Z[(size_t)i * n + j] * Z[(size_t)i * n + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (!(nrm > (R)0) || !isfinite(nrm)) {
      if (lane == 0) atomicExch(info, 1);
      nrm = 1;
    }
    const R inv = (R)1 / sqrt(nrm);
    for (int i = lane; i < n; i += 32) Z[(size_t)i * n + j] *= inv;
    __syncwarp();
  }
}

// -------------------------------------------------------------------------------------------------
// 4. back-transformation: V[:, c] = H_0 H_1 ... H_{n-2} D^H Z[:, c]; one warp per column. Element i of
// u_j is at U[j sj + i si].
// -------------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_backtransform(int n, const cplx<R>* __restrict__ U, size_t sj, size_t si,
                                                       const R* __restrict__ tau, const cplx<R>* __restrict__ ph,
                                                       const R* __restrict__ Z, cplx<R>* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cpb = blockDim.x >> 5;  // columns per CTA
  cplx<R>* vc = reinterpret_cast<cplx<R>*>(smem_raw);  // n x cpb
  const int lane = threadIdx.x & 31, wc = threadIdx.x >> 5;
  const int col = blockIdx.x * cpb + wc;
  if (col >= n) return;
  for (int i = lane; i < n; i += 32) vc[(size_t)i * cpb + wc] = cscale(cconj(ph[i]), Z[(size_t)i * n + col]);
  __syncwarp();
  for (int j = n - 2; j >= 0; --j) {
    const R t = tau[j];
    if (t == (R)0) continue;
    const int m = n - j - 1;
    cplx<R> s = mk<R>(0, 0);
    const cplx<R>* u = U + (size_t)j * sj;
    for (int i = lane; i < m; i += 32) s = cadd(s, cmul(cconj(u[i * si]), vc[(size_t)(j + 1 + i) * cpb + wc]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    s = cscale(s, t);
    for (int i = lane; i < m; i += 32) {
      cplx<R>& v = vc[(size_t)(j + 1 + i) * cpb + wc];
      v = csub(v, cmul(u[i * si], s));
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) V[(size_t)i * n + col] = vc[(size_t)i * cpb + wc];
}

// The same with every reflector in shared memory (when n^2 values of cplx<R> fit): U rows u_j at
// Us[j * n + i]; one warp per column, blockDim / 32 columns per CTA.
template <typename R>
__global__ void __launch_bounds__(512) k_backtransform_s(int n, const cplx<R>* __restrict__ U, const R* __restrict__ tau,
                                                         const cplx<R>* __restrict__ ph, const R* __restrict__ Z,
                                                         cplx<R>* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cpb = blockDim.x >> 5;
  cplx<R>* Us = reinterpret_cast<cplx<R>*>(smem_raw);  // n x n (row j = u_j, m = n - j - 1 entries used)
  cplx<R>* vc = Us + (size_t)n * n;                   // cpb x n: column wc of this CTA contiguous
  R* ts = reinterpret_cast<R*>(vc + (size_t)n * cpb);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) Us[i] = U[i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) ts[i] = tau[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wc = threadIdx.x >> 5;
  const int col = blockIdx.x * cpb + wc;
  if (col >= n) return;
  for (int i = lane; i < n; i += 32) vc[(size_t)wc * n + i] = cscale(cconj(ph[i]), Z[(size_t)i * n + col]);
  __syncwarp();
  for (int j = n - 2; j >= 0; --j) {
    const R t = ts[j];
    if (t == (R)0) continue;
    const int m = n - j - 1;
    cplx<R> sv = mk<R>(0, 0);
    const cplx<R>* u = Us + (size_t)j * n;
    for (int i = lane; i < m; i += 32) sv = cadd(sv, cmul(cconj(u[i]), vc[(size_t)wc * n + j + 1 + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
      sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
    }
    sv = cscale(sv, t);
    for (int i = lane; i < m; i += 32) {
      cplx<R>& vv = vc[(size_t)wc * n + j + 1 + i];
      vv = csub(vv, cmul(u[i], sv));
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) V[(size_t)i * n + col] = vc[(size_t)wc * n + i];
}

// Blocked back-transformation (compact WY form, forward accumulation): the reflectors in blocks of
// kWY, H_j0 ... H_j0+k-1 = I - V T V^H with T upper triangular, T_ii = tau_i and
// T(0:i, i) = -tau_i T(0:i, 0:i) V(:, 0:i)^H v_i; then V_eig = Q_0 Q_1 ... (D^H Z), each block applied as
// Z -= V (T (V^H Z)), three small products instead of k dependent reflector steps per column.
static const int kWY = 16;

// T of every block (one CTA of 256 threads per block): Tb[b] is kWY x kWY, row-major
template <typename R>
__global__ void __launch_bounds__(256) k_wy_t(int n, const cplx<R>* __restrict__ U, const R* __restrict__ tau,
                                              cplx<R>* __restrict__ Tb) {
  __shared__ cplx<R> Gm[kWY][kWY + 1];  // G(i, l) = v_i^H v_l, i < l
  __shared__ cplx<R> T[kWY][kWY + 1];
  const int b = blockIdx.x, j0 = b * kWY, nbk = min(kWY, n - 1 - j0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // v_j[r] = U[j n + r - j - 1] for r > j: the overlap of v_i and v_l (i < l) is r > j0 + l
  for (int pr = warp; pr < kWY * kWY; pr += nwarp) {
    const int i = pr / kWY, l = pr - i * kWY;
    if (i >= l || l >= nbk) continue;
    const int ji = j0 + i, jl = j0 + l;
    cplx<R> acc = mk<R>(0, 0);
    for (int r = jl + 1 + lane; r < n; r += 32)
      acc = cadd(acc, cmul(cconj(U[(size_t)ji * n + (r - ji - 1)]), U[(size_t)jl * n + (r - jl - 1)]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) Gm[i][l] = acc;
  }
  for (int idx = threadIdx.x; idx < kWY * kWY; idx += blockDim.x) {
    const int i = idx / kWY, l = idx - i * kWY;
    T[i][l] = mk<R>(i == l && i < nbk ? tau[j0 + i] : (R)0, 0);
  }
  __syncthreads();
  if (warp == 0) {
    for (int l = 1; l < nbk; ++l) {  // T(i, l) = -tau_l sum_{k = i}^{l-1} T(i, k) G(k, l), lane i < l
      cplx<R> acc = mk<R>(0, 0);
      if (lane < l)
        for (int k = lane; k < l; ++k) acc = cadd(acc, cmul(T[lane][k], Gm[k][l]));
      __syncwarp();
      if (lane < l) T[lane][l] = cscale(acc, -tau[j0 + l]);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kWY * kWY; idx += blockDim.x)
    Tb[(size_t)b * kWY * kWY + idx] = T[idx / kWY][idx % kWY];
}

// V[:, c] for the CG columns c0.. of this CTA: Zc = D^H Z[:, c], then every block from the last to the
// first: W = V_b^H Zc (kWY x CG), W = T_b W, Zc -= V_b W. V_b staged in shared memory per block.
template <typename R, int CG>
__global__ void __launch_bounds__(256) k_wy_apply(int n, const cplx<R>* __restrict__ U, const cplx<R>* __restrict__ Tb,
                                                  const cplx<R>* __restrict__ ph, const R* __restrict__ Z,
                                                  cplx<R>* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Zc = reinterpret_cast<cplx<R>*>(smem_raw);  // n x CG
  cplx<R>* Vs = Zc + (size_t)n * CG;                   // kWY x n: Vs[i][r] = v_{j0+i}[r] (0 for r <= j0 + i)
  __shared__ cplx<R> W[kWY][CG], W2[kWY][CG], Ts[kWY][kWY];
  const int c0 = blockIdx.x * CG, nc = min(CG, n - c0);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < n * CG; idx += blockDim.x) {
    const int r = idx / CG, cc = idx - r * CG;
    Zc[idx] = cc < nc ? cscale(cconj(ph[r]), Z[(size_t)r * n + c0 + cc]) : mk<R>(0, 0);
  }
  const int nblk = (n - 1 + kWY - 1) / kWY;
  for (int b = nblk - 1; b >= 0; --b) {
    const int j0 = b * kWY, nbk = min(kWY, n - 1 - j0);
    __syncthreads();  // Zc complete; the previous block's Vs, W2 no longer read
    for (int idx = tid; idx < kWY * n; idx += blockDim.x) {
      const int i = idx / n, r = idx - i * n, j = j0 + i;
      Vs[idx] = (i < nbk && r > j) ? U[(size_t)j * n + (r - j - 1)] : mk<R>(0, 0);
    }
    for (int idx = tid; idx < kWY * kWY; idx += blockDim.x)
      Ts[idx / kWY][idx % kWY] = Tb[(size_t)b * kWY * kWY + idx];
    __syncthreads();
    for (int idx = tid; idx < kWY * CG; idx += blockDim.x) {  // W = V_b^H Zc
      const int i = idx / CG, cc = idx - i * CG;
      cplx<R> acc = mk<R>(0, 0);
      for (int r = j0 + i + 1; r < n; ++r) acc = cadd(acc, cmul(cconj(Vs[i * n + r]), Zc[r * CG + cc]));
      W[i][cc] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < kWY * CG; idx += blockDim.x) {  // W2 = T W (T upper triangular)
      const int i = idx / CG, cc = idx - i * CG;
      cplx<R> acc = mk<R>(0, 0);
      for (int k = i; k < kWY; ++k) acc = cadd(acc, cmul(Ts[i][k], W[k][cc]));
      W2[i][cc] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < (n - j0 - 1) * CG; idx += blockDim.x) {  // Zc -= V_b W2 (rows r > j0)
      const int r = j0 + 1 + idx / CG, cc = idx % CG;
      cplx<R> acc = mk<R>(0, 0);
#pragma unroll 4
      for (int i = 0; i < kWY; ++i) acc = cadd(acc, cmul(Vs[i * n + r], W2[i][cc]));
      Zc[r * CG + cc] = csub(Zc[r * CG + cc], acc);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * CG; idx += blockDim.x) {
    const int r = idx / CG, cc = idx - r * CG;
    if (cc < nc) V[(size_t)r * n + c0 + cc] = Zc[idx];
  }
}

// CTAs of a cooperative launch of `kernel` with `threads` threads and `smem` bytes: at most `cap`,
// and no more than can be co-resident.
int coop_grid(Ctx* c, const void* kernel, int threads, size_t smem, int cap, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  PARO_CU(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PARO_CU(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  int g = per_sm * sms;
  if (g > cap) g = cap;
  if (g < 1) return fail(c, PARO_ERR_ARG, "cooperative kernel cannot be resident");
  *grid = g;
  return PARO_OK;
}

// Cluster shape for k_tridiag_cluster: 16 CTAs where the device allows a cluster of that size with the
// needed shared memory, else 8; *cls = 0 when neither fits (the grid-barrier kernel is used).
static int tridiag_cluster_shape(Ctx* c, int n, int* cls, int* thr, size_t* smem) {
  *cls = 0;
  PARO_CU(c, cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  PARO_CU(c, cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  for (int C : {16, 8}) {
    const int R = (n + C - 1) / C;
    const size_t sm = ((size_t)R * n + 6 * (size_t)n) * sizeof(double2) + 2 * sizeof(double);
    if (sm > 200 * 1024) continue;
    const int warps = R < 4 ? 4 : (R > 32 ? 32 : R);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_tridiag_cluster, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters >= 1) {
      *cls = C;
      *thr = 32 * warps;
      *smem = sm;
      return PARO_OK;
    }
  }
  return PARO_OK;
}

// Inverse iteration for the n eigenvectors of the tridiagonal (d, e) at the ascending eigenvalues w
// into Z (column j = vector j); info set if a vector vanished.
template <typename R>
int invit(Ctx* c, int n, const R* d, const R* e, const R* w, R* Z, int* info) {
  const bool f64 = sizeof(R) == 8;
  R* lam = static_cast<R*>(ws_get(c, f64 ? "invit_lam64" : "invit_lam32", (size_t)(n + 1) * sizeof(R)));
  int* cst = static_cast<int*>(ws_get(c, "invit_cst", (size_t)(n + 2) * sizeof(int)));
  if (!lam || !cst) return PARO_ERR_CUDA;
  int* nclu = cst + n + 1;
  R* tiny = lam + n;
  k_invit_prep<R><<<1, 32, 0, c->stream>>>(n, d, e, w, lam, cst, nclu, tiny);
  PARO_LAUNCH(c, "k_invit_prep");
  const size_t per = (size_t)n * (5 * sizeof(R) + 1);
  int E = (int)std::min<size_t>(32, (200 * 1024) / per);
  if (E < 1) return fail(c, PARO_ERR_ARG, "inverse iteration: n too large");
  const size_t sm = per * E;
  PARO_CU(c, cudaFuncSetAttribute(k_invit_solve<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  R* fac = static_cast<R*>(ws_get(c, f64 ? "invit_fac64" : "invit_fac32", (size_t)4 * n * n * sizeof(R)));
  unsigned char* swg = static_cast<unsigned char*>(ws_get(c, "invit_sw", (size_t)n * n));
  if (!fac || !swg) return PARO_ERR_CUDA;
  for (int it = 0; it < 3; ++it) {
    k_invit_solve<R><<<(n + E - 1) / E, E, sm, c->stream>>>(n, d, e, lam, tiny, Z, it == 0 ? 1 : 0, fac, swg,
                                                            info);
    PARO_LAUNCH(c, "k_invit_solve");
    k_invit_mgs<R><<<(n + 3) / 4, 128, 0, c->stream>>>(n, Z, cst, nclu, info);
    PARO_LAUNCH(c, "k_invit_mgs");
  }
  return PARO_OK;
}
template int invit<double>(Ctx*, int, const double*, const double*, const double*, double*, int*);
template int invit<float>(Ctx*, int, const float*, const float*, const float*, float*, int*);

// FP32 multisection, inverse iteration and back-transformation of the mixed-precision solver
// (k_eigh_mixed.cu): w ascending eigenvalues of (d, e), V[:, j] the eigenvector of the Hermitian matrix
// whose reflectors are the rows of U.
int eigh_fp32_pieces(Ctx* c, int n, const float* d, const float* e, float* w, const float2* U, const float* tau,
                     const float2* ph, float* Z, float2* V, int* info) {
  cudaEvent_t ev = prof_begin(c);
  k_bisect<float><<<(n + 3) / 4, 128, (size_t)2 * n * sizeof(float), c->stream>>>(n, d, e, w);
  PARO_LAUNCH(c, "k_bisect");
  prof_end(c, "eigh32_bisect", ev);
  ev = prof_begin(c);
  int st = invit<float>(c, n, d, e, w, Z, info);
  if (st) return st;
  prof_end(c, "eigh32_invit", ev);
  ev = prof_begin(c);
  {  // blocked (compact WY) back-transformation
    const int nblk = (n - 1 + kWY - 1) / kWY;
    constexpr int CG = 8;
    const size_t smw = ((size_t)n * CG + (size_t)kWY * n) * sizeof(float2);
    float2* Tb = static_cast<float2*>(ws_get(c, "wy_T32", (size_t)std::max(nblk, 1) * kWY * kWY * sizeof(float2)));
    if (!Tb) return PARO_ERR_CUDA;
    if (smw <= 200 * 1024 && n >= 2) {
      k_wy_t<float><<<nblk, 256, 0, c->stream>>>(n, U, tau, Tb);
      PARO_LAUNCH(c, "k_wy_t");
      PARO_CU(c, cudaFuncSetAttribute(k_wy_apply<float, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
      k_wy_apply<float, CG><<<(n + CG - 1) / CG, 256, smw, c->stream>>>(n, U, Tb, ph, Z, V);
      PARO_LAUNCH(c, "k_wy_apply");
      prof_end(c, "eigh32_backtransform", ev);
      return PARO_OK;
    }
  }
  const int cpb = 4;
  const size_t sms = ((size_t)n * n + (size_t)n * cpb) * sizeof(float2) + (size_t)n * sizeof(float);
  if (sms <= 220 * 1024) {  // reflectors in shared memory
    PARO_CU(c, cudaFuncSetAttribute(k_backtransform_s<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms));
    k_backtransform_s<float><<<(n + cpb - 1) / cpb, 32 * cpb, sms, c->stream>>>(n, U, tau, ph, Z, V);
    PARO_LAUNCH(c, "k_backtransform_s");
    prof_end(c, "eigh32_backtransform", ev);
    return PARO_OK;
  }
  const int cpb2 = 2;
  const size_t sm4 = (size_t)n * cpb2 * sizeof(float2);
  PARO_CU(c, cudaFuncSetAttribute(k_backtransform<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4));
  k_backtransform<float><<<(n + cpb2 - 1) / cpb2, 32 * cpb2, sm4, c->stream>>>(n, U, (size_t)n, 1, tau, ph, Z, V);
  PARO_LAUNCH(c, "k_backtransform");
  prof_end(c, "eigh32_backtransform", ev);
  return PARO_OK;
}

int eigh(Ctx* c, int n, const double2* a, double* w, double2* v) {
  if (n < 1 || n > 1024) return fail(c, PARO_ERR_ARG, "eigh: n must be in [1, 1024]");
  double2* A = static_cast<double2*>(ws_get(c, "eigh_A", (size_t)n * n * sizeof(double2)));
  double* Z = static_cast<double*>(ws_get(c, "eigh_Z", (size_t)n * n * sizeof(double)));
  double* dt = static_cast<double*>(ws_get(c, "eigh_dt", (size_t)n * 4 * sizeof(double)));
  double2* cw = static_cast<double2*>(ws_get(c, "eigh_cw", (size_t)n * 4 * sizeof(double2)));
  int* flags = static_cast<int*>(ws_get(c, "eigh_flags", 16 * sizeof(int)));
  if (!A || !Z || !dt || !cw || !flags) return PARO_ERR_CUDA;
  double *d = dt, *e = dt + n, *tau = dt + 2 * n, *sc = dt + 3 * n;
  double2 *ph = cw, *ecx = cw + n, *ub = cw + 2 * n, *pb = cw + 3 * n;
  unsigned* bar = reinterpret_cast<unsigned*>(flags);
  int* err = flags + 2;
  int* info = flags + 3;
  PARO_CU(c, cudaMemsetAsync(flags, 0, 16 * sizeof(int), c->stream));
  // Householder vectors: row j of A (cluster path) or column j of the work copy (grid path)
  const double2* Uh = A + n;
  size_t usj = (size_t)n + 1, usi = (size_t)n;
  int cls = 0, thr = 0, st;
  size_t smc = 0;
  if ((st = tridiag_cluster_shape(c, n, &cls, &thr, &smc))) return st;
  cudaEvent_t ev = prof_begin(c);
  if (cls > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cls;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cls);
    cfg.blockDim = dim3(thr);
    cfg.dynamicSmemBytes = smc;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    PARO_CU(c, cudaLaunchKernelEx(&cfg, k_tridiag_cluster, n, a, A, d, e, ph, tau, ecx));
    ++c->launches;
    Uh = A;
    usj = (size_t)n;
    usi = 1;
    prof_end(c, "k_tridiag_cluster", ev);
  } else {
    k_herm_full<<<(n * n + 255) / 256, 256, 0, c->stream>>>(n, a, A);
    PARO_LAUNCH(c, "k_herm_full");
    const size_t sm1 = (size_t)2 * n * sizeof(double2);
    int grid = 1;
    if ((st = coop_grid(c, (const void*)k_tridiag, 256, sm1, 64, &grid))) return st;
    int nn = n;
    void* args[] = {&nn, &A, &d, &e, &ph, &tau, &ecx, &ub, &pb, &sc, &bar, &err};
    PARO_CU(c, cudaLaunchCooperativeKernel((const void*)k_tridiag, dim3(grid), dim3(256), args, sm1, c->stream));
    ++c->launches;
    prof_end(c, "k_tridiag", ev);
  }
  ev = prof_begin(c);
  k_bisect<double><<<(n + 3) / 4, 128, (size_t)2 * n * sizeof(double), c->stream>>>(n, d, e, w);
  PARO_LAUNCH(c, "k_bisect");
  prof_end(c, "k_bisect", ev);
  ev = prof_begin(c);
  if ((st = invit<double>(c, n, d, e, w, Z, info))) return st;
  prof_end(c, "k_invit", ev);
  ev = prof_begin(c);
  const int cpb = 2;
  const size_t sm4 = (size_t)n * cpb * sizeof(double2);
  PARO_CU(c, cudaFuncSetAttribute(k_backtransform<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4));
  k_backtransform<double><<<(n + cpb - 1) / cpb, 32 * cpb, sm4, c->stream>>>(n, Uh, usj, usi, tau, ph, Z, v);
  PARO_LAUNCH(c, "k_backtransform");
  prof_end(c, "k_backtransform", ev);
  int h[2] = {0, 0};
  PARO_CU(c, cudaMemcpyAsync(h, flags + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  if (h[0]) return fail(c, PARO_ERR_TIMEOUT, "eigh: grid barrier wait gave up");
  if (h[1]) return fail(c, PARO_ERR_NOT_CONVERGED, "eigh: inverse iteration produced a zero or non-finite vector");
  return PARO_OK;
}

}  // namespace paro
