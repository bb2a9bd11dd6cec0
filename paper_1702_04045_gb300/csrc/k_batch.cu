// Batched ParO over many independent small problems: the k-points of one cell and/or separate cells
// with uneven plane-wave counts and FFT grids ("two-level parallelism": every orbital of every
// problem is an independent source problem, Algorithm 1 step 3, and the projection step 4 is local to
// its problem).
//
//  * H psi: one persistent kernel per apply over flat work lists of every problem's orbitals, in three
//    phases: z-FFTs of stick groups (and the projections per orbital), one unit per (orbital, z-plane)
//    for the 2D FFTs and V_eff(r), and z-FFTs back with the gather, kinetic and projector terms. The
//    phases are separated by bounded grid barriers of a cooperative launch, or by kernel boundaries
//    (three launches) when that is faster; the stick buffers stay in L2.
//  * PCG: the batched kernels of the per-context solver, over a ragged list of bands (per-band plane-wave
//    count and offset), with per-band convergence masks on the device and a fixed number of steps.
//  * projection: per problem (n_bands <= 64) Gram and H_sub by split-K products, Cholesky and
//    triangular inverse in one CTA, a cyclic Jacobi eigensolver (parallel round-robin ordering) in one CTA,
//    and the rotations.
//  * one ParO step is captured once into a CUDA graph and replayed; nothing in it waits on the host.
//  * the H psi form (one cooperative launch or three) and its persistent grid are picked by timing the
//    candidates on the batch's own problems when the batch is created.
#include <algorithm>
#include <array>
#include <cfloat>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "jacobi_small.cuh"
#include "paro_ctx.h"

namespace paro {

static const int kBMaxBands = 64;
static const int kBChunk = 1024;  // plane waves per CTA in the batched vector kernels
static const int kBSlice = 512;   // K slice of the batched Gram / H_sub products

// Per problem (one k-point of one context), device-visible.
struct ProbDev {
  int npw, ncol, nxr, nb, N1, N2, N3, nproj;
  long long off;   // first element of the problem's rows in the batch vectors
  long long soff;  // first element of the problem's stick buffers (nb x N3 x ncol)
  long long dpoff; // first element of the problem's scaled projections (nb x nproj)
  int band0;       // first band of the problem in the flat band list
  int pad;
  FftPlan plan[3];
  const int *col_x, *col_y, *col_off, *g_col, *g_z, *xrows;
  const double* kin;
  const float* kin32;
  const double* vplane;
  const float* vplane32;
  const double2* tw64[3];
  const float2* tw32[3];
  const double2* beta;
  const float2* beta32;
  const double* dvec;
};

template <typename T> __device__ __forceinline__ const cplx<T>* pd_tw(const ProbDev& p, int a);
template <> __device__ __forceinline__ const double2* pd_tw<double>(const ProbDev& p, int a) { return p.tw64[a]; }
template <> __device__ __forceinline__ const float2* pd_tw<float>(const ProbDev& p, int a) { return p.tw32[a]; }
template <typename T> __device__ __forceinline__ const T* pd_kin(const ProbDev& p);
template <> __device__ __forceinline__ const double* pd_kin<double>(const ProbDev& p) { return p.kin; }
template <> __device__ __forceinline__ const float* pd_kin<float>(const ProbDev& p) { return p.kin32; }
template <typename T> __device__ __forceinline__ const T* pd_v(const ProbDev& p);
template <> __device__ __forceinline__ const double* pd_v<double>(const ProbDev& p) { return p.vplane; }
template <> __device__ __forceinline__ const float* pd_v<float>(const ProbDev& p) { return p.vplane32; }
template <typename T> __device__ __forceinline__ const cplx<T>* pd_beta(const ProbDev& p);
template <> __device__ __forceinline__ const double2* pd_beta<double>(const ProbDev& p) { return p.beta; }
template <> __device__ __forceinline__ const float2* pd_beta<float>(const ProbDev& p) { return p.beta32; }

// Work-unit shapes, chosen per batch by the autotuner: sg sticks per z-FFT unit, and z-planes per plane
// unit enough that one unit's FFT stages cover about ppt points (at most 4 planes)
__host__ __device__ __forceinline__ int planes_per_unit(int N1, int N2, int ppt) {
  const int pb = ppt / (N1 * N2);
  return pb < 1 ? 1 : (pb > 4 ? 4 : pb);
}

// shared memory of one work unit (in elements of cplx<T>): the larger of a stick group's lines and a
// plane, plus the three twiddle tables
static size_t unit_elems(const ProbDev& p, int sg, int ppt) {
  const size_t lines = (size_t)sg * (p.N3 + 1), plane = (size_t)p.N1 * p.N2 * planes_per_unit(p.N1, p.N2, ppt);
  return (lines > plane ? lines : plane) + p.N1 + p.N2 + p.N3;
}

// ------------------------------------------------------------------------------------------------
// H psi of every (problem, band) item in one persistent cooperative launch: Y = (H - shift_p) X,
// shift_p = sigma_p when `shifted`. Three phases over flat work lists, separated by bounded grid
// barriers; the stick buffers S (plane-major per item) and the scaled projections DP stay in L2.
//   phase 1: (item, stick group) - scatter the group's coefficients on lines of N3 points and
//            inverse-FFT them along z into S; (item, -1) - D_j (beta_j^H c) for the item's projectors
//   phase 2: (item, z) - the plane: inverse FFT along y (rows with sticks) and x, times V(z)/N, forward
//            FFT along x and y, back into S
//   phase 3: (item, stick group) - forward FFT along z, gather, add (|k+G|^2/2 - shift) c_G and the
//            projector term sum_j beta_j(G) DP_j
// ------------------------------------------------------------------------------------------------
struct HpsiLists {
  const int2* u1; int n1;  // (item, group or -1)
  const int2* u2; int n2;  // (item, z)
  const int2* u3; int n3;  // (item, group)
  int sg, ppt;             // sticks per z-FFT unit; plane points per plane unit
};

// PH = 0: all three phases in one cooperative launch (grid barriers between them); PH = 1, 2, 3: one
// phase per launch (the kernel boundary orders them).
template <typename T, int PH>
__global__ void __launch_bounds__(256, PH == 0 ? 1 : 2) k_hpsi_batch(const ProbDev* __restrict__ probs, const int2* __restrict__ items,
                                                    HpsiLists L, const cplx<T>* __restrict__ X, cplx<T>* __restrict__ Y,
                                                    cplx<T>* __restrict__ S, cplx<T>* __restrict__ DP,
                                                    const int* __restrict__ active, const double* __restrict__ sigma,
                                                    int shifted, unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ProbDev pd;
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // returns false when the unit's item is inactive (the whole CTA skips it)
  auto begin_unit = [&](int2 u) -> bool {
    __syncthreads();
    if (threadIdx.x == 0) pd = probs[items[u.x].x];
    __syncthreads();
    return active == nullptr || active[pd.band0 + items[u.x].y] != 0;
  };
  // ---- phase 1
  if (PH == 0 || PH == 1)
  for (int ui = blockIdx.x; ui < L.n1; ui += gridDim.x) {
    const int2 u = L.u1[ui];
    if (!begin_unit(u)) continue;
    const int b = items[u.x].y, npw = pd.npw, ncol = pd.ncol, N3 = pd.N3;
    const cplx<T>* x = X + pd.off + (size_t)b * npw;
    if (u.y < 0) {  // projections
      const cplx<T>* beta = pd_beta<T>(pd);
      cplx<T>* dp = DP + pd.dpoff + (size_t)b * pd.nproj;
      for (int j = warp; j < pd.nproj; j += nwarp) {
        const cplx<T>* bj = beta + (size_t)j * npw;
        T sx = 0, sy = 0;
        for (int g = lane; g < npw; g += 32) {
          const cplx<T> bv = bj[g], c = x[g];
          sx += bv.x * c.x + bv.y * c.y;  // conj(beta) c
          sy += bv.x * c.y - bv.y * c.x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sx += __shfl_xor_sync(0xffffffffu, sx, o);
          sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) dp[j] = mk<T>((T)(pd.dvec[j] * sx), (T)(pd.dvec[j] * sy));
      }
      continue;
    }
    const int c0 = u.y * L.sg, ncb = min(L.sg, ncol - c0), ls = N3 + 1;
    cplx<T>* tz = buf;
    cplx<T>* line = tz + N3;
    for (int i = threadIdx.x; i < N3; i += blockDim.x) tz[i] = pd_tw<T>(pd, 2)[i];
    for (int i = threadIdx.x; i < ncb * ls; i += blockDim.x) line[i] = mk<T>(0, 0);
    __syncthreads();
    const int g0 = pd.col_off[c0], g1 = pd.col_off[c0 + ncb];
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) line[(pd.g_col[g] - c0) * ls + pd.g_z[g]] = x[g];
    __syncthreads();
    fft_lines<T, true, false>(line, pd.plan[2], ncb, 1, LinesDirect{ls}, tz);
    cplx<T>* Sb = S + pd.soff + (size_t)b * N3 * ncol;
    for (int i = threadIdx.x; i < N3 * ncb; i += blockDim.x) {
      const int z = i / ncb, cc = i - z * ncb;
      Sb[(size_t)z * ncol + c0 + cc] = line[cc * ls + z];
    }
  }
  if (PH == 0 && !grid_barrier(bar, err)) return;
  // ---- phase 2
  if (PH == 0 || PH == 2)
  for (int ui = blockIdx.x; ui < L.n2; ui += gridDim.x) {
    const int2 u = L.u2[ui];
    if (!begin_unit(u)) continue;
    const int b = items[u.x].y, N1 = pd.N1, N2 = pd.N2, ncol = pd.ncol, PS = N1 * N2;
    const int z0 = u.y, np = min(planes_per_unit(N1, N2, L.ppt), pd.N3 - z0);
    cplx<T>* tx = buf;
    cplx<T>* ty = tx + N1;
    cplx<T>* P = ty + N2;  // np planes
    for (int i = threadIdx.x; i < N1; i += blockDim.x) tx[i] = pd_tw<T>(pd, 0)[i];
    for (int i = threadIdx.x; i < N2; i += blockDim.x) ty[i] = pd_tw<T>(pd, 1)[i];
    for (int i = threadIdx.x; i < np * PS; i += blockDim.x) P[i] = mk<T>(0, 0);
    __syncthreads();
    cplx<T>* Sz = S + pd.soff + ((size_t)b * pd.N3 + z0) * ncol;
    for (int i = threadIdx.x; i < np * ncol; i += blockDim.x) {
      const int q = i / ncol, c = i - q * ncol;
      P[q * PS + pd.col_x[c] * N2 + pd.col_y[c]] = Sz[(size_t)q * ncol + c];
    }
    __syncthreads();
    fft_lines<T, true, false>(P, pd.plan[1], np * pd.nxr, 1, LinesPlanes{pd.xrows, pd.nxr, N2, PS}, ty);
    fft_lines<T, true, true>(P, pd.plan[0], np * N2, N2, LinesPlanes{nullptr, N2, 1, PS}, tx);
    const T* Vz = pd_v<T>(pd) + (size_t)z0 * PS;
    for (int i = threadIdx.x; i < np * PS; i += blockDim.x) P[i] = cscale(P[i], Vz[i]);
    __syncthreads();
    fft_lines<T, false, true>(P, pd.plan[0], np * N2, N2, LinesPlanes{nullptr, N2, 1, PS}, tx);
    fft_lines<T, false, false>(P, pd.plan[1], np * pd.nxr, 1, LinesPlanes{pd.xrows, pd.nxr, N2, PS}, ty);
    for (int i = threadIdx.x; i < np * ncol; i += blockDim.x) {
      const int q = i / ncol, c = i - q * ncol;
      Sz[(size_t)q * ncol + c] = P[q * PS + pd.col_x[c] * N2 + pd.col_y[c]];
    }
  }
  if (PH == 0 && !grid_barrier(bar, err)) return;
  // ---- phase 3
  if (PH == 0 || PH == 3)
  for (int ui = blockIdx.x; ui < L.n3; ui += gridDim.x) {
    const int2 u = L.u3[ui];
    if (!begin_unit(u)) continue;
    const int b = items[u.x].y, npw = pd.npw, ncol = pd.ncol, N3 = pd.N3, np = pd.nproj;
    const int c0 = u.y * L.sg, ncb = min(L.sg, ncol - c0), ls = N3 + 1;
    cplx<T>* tz = buf;
    cplx<T>* line = tz + N3;
    for (int i = threadIdx.x; i < N3; i += blockDim.x) tz[i] = pd_tw<T>(pd, 2)[i];
    const cplx<T>* Sb = S + pd.soff + (size_t)b * N3 * ncol;
    for (int i = threadIdx.x; i < N3 * ncb; i += blockDim.x) {
      const int z = i / ncb, cc = i - z * ncb;
      line[cc * ls + z] = Sb[(size_t)z * ncol + c0 + cc];
    }
    __syncthreads();
    fft_lines<T, false, false>(line, pd.plan[2], ncb, 1, LinesDirect{ls}, tz);
    const cplx<T>* x = X + pd.off + (size_t)b * npw;
    cplx<T>* y = Y + pd.off + (size_t)b * npw;
    const cplx<T>* dp = DP + pd.dpoff + (size_t)b * np;
    const cplx<T>* beta = pd_beta<T>(pd);
    const T sh = shifted ? (T)sigma[items[u.x].x] : (T)0;
    const T* kin = pd_kin<T>(pd);
    const int g0 = pd.col_off[c0], g1 = pd.col_off[c0 + ncb];
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      const cplx<T> v = line[(pd.g_col[g] - c0) * ls + pd.g_z[g]], c = x[g];
      const T t = kin[g] - sh;
      T hx = v.x + t * c.x, hy = v.y + t * c.y;
      for (int j = 0; j < np; ++j) {
        const cplx<T> bv = beta[(size_t)j * npw + g], d = dp[j];
        hx += bv.x * d.x - bv.y * d.y;
        hy += bv.x * d.y + bv.y * d.x;
      }
      y[g] = mk<T>(hx, hy);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// batched PCG over the flat band list (same recurrences and stopping test as the per-context solver)
// ------------------------------------------------------------------------------------------------
struct BandMap {
  const int* prob;         // problem of flat band gb
  const int* row;          // band index inside its problem
  const ProbDev* probs;
};

template <typename T>
__global__ void __launch_bounds__(256) k_bpcg_init(BandMap bm, int nch, const cplx<T>* __restrict__ bvec,
                                                   const cplx<T>* __restrict__ ax, cplx<T>* __restrict__ r,
                                                   cplx<T>* __restrict__ p, const double* __restrict__ pshift,
                                                   double* __restrict__ prz, double* __restrict__ prr) {
  __shared__ double red[32];
  const int gb = blockIdx.y, ch = blockIdx.x;
  const int pi = bm.prob[gb];
  const ProbDev& P = bm.probs[pi];
  const int npw = P.npw;
  const size_t o = P.off + (size_t)bm.row[gb] * npw;
  const T* kin = pd_kin<T>(P);
  const T ps = (T)pshift[pi];
  double rz = 0.0, rr = 0.0;
  const int g0 = ch * kBChunk, g1 = min(npw, g0 + kBChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const cplx<T> rv = csub(bvec[o + g], ax[o + g]);
    const T m = (T)1 / (kin[g] + ps);
    r[o + g] = rv;
    p[o + g] = cscale(rv, m);
    const double q = (double)rv.x * rv.x + (double)rv.y * rv.y;
    rr += q;
    rz += q * (double)m;
  }
  rz = block_sum(rz, red);
  if (threadIdx.x == 0) prz[(size_t)gb * nch + ch] = rz;
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) prr[(size_t)gb * nch + ch] = rr;
}

__global__ void k_bpcg_band_init(int nbt, int nch, const double* __restrict__ prz, const double* __restrict__ prr,
                                 double* __restrict__ rz, double* __restrict__ r0n, int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbt) return;
  double a = 0.0, q = 0.0;
  for (int ch = 0; ch < nch; ++ch) {
    a += prz[(size_t)b * nch + ch];
    q += prr[(size_t)b * nch + ch];
  }
  rz[b] = a;
  r0n[b] = sqrt(q);
  active[b] = q > 0.0 ? 1 : 0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bpcg_dot(BandMap bm, int nch, const cplx<T>* __restrict__ p,
                                                  const cplx<T>* __restrict__ ap, const int* __restrict__ active,
                                                  double* __restrict__ part) {
  __shared__ double red[32];
  const int gb = blockIdx.y, ch = blockIdx.x;
  if (!active[gb]) return;
  const ProbDev& P = bm.probs[bm.prob[gb]];
  const int npw = P.npw;
  const size_t o = P.off + (size_t)bm.row[gb] * npw;
  double s = 0.0;
  const int g0 = ch * kBChunk, g1 = min(npw, g0 + kBChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const cplx<T> u = p[o + g], v = ap[o + g];
    s += (double)u.x * v.x + (double)u.y * v.y;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(size_t)gb * nch + ch] = s;
}

__global__ void k_bpcg_alpha(int nbt, int nch, const double* __restrict__ part, const double* __restrict__ rz,
                             const int* __restrict__ active, double* __restrict__ alpha, int* __restrict__ bad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbt) return;
  if (!active[b]) {
    alpha[b] = 0.0;
    return;
  }
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[(size_t)b * nch + ch];
  if (!(s > 0.0) || !isfinite(s)) {
    atomicExch(bad, b + 1);
    alpha[b] = 0.0;
    return;
  }
  alpha[b] = rz[b] / s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bpcg_update(BandMap bm, int nch, cplx<T>* __restrict__ x,
                                                     cplx<T>* __restrict__ r, const cplx<T>* __restrict__ p,
                                                     const cplx<T>* __restrict__ ap, const double* __restrict__ pshift,
                                                     const double* __restrict__ alpha, const int* __restrict__ active,
                                                     double* __restrict__ prr, double* __restrict__ prz,
                                                     cplx<T>* __restrict__ hx, const double* __restrict__ sigma) {
  __shared__ double red[32];
  const int gb = blockIdx.y, ch = blockIdx.x;
  if (!active[gb]) return;
  const int pi = bm.prob[gb];
  const ProbDev& P = bm.probs[pi];
  const int npw = P.npw;
  const size_t o = P.off + (size_t)bm.row[gb] * npw;
  const T* kin = pd_kin<T>(P);
  const T ps = (T)pshift[pi];
  const T a = (T)alpha[gb];
  const T sg = hx ? (T)sigma[pi] : (T)0;
  double rr = 0.0, rz = 0.0;
  const int g0 = ch * kBChunk, g1 = min(npw, g0 + kBChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const cplx<T> pv = p[o + g], av = ap[o + g];
    cplx<T> xv = x[o + g], rv = r[o + g];
    xv.x += a * pv.x; xv.y += a * pv.y;
    rv.x -= a * av.x; rv.y -= a * av.y;
    x[o + g] = xv;
    r[o + g] = rv;
    if (hx) {  // H x follows x: H p = ap + sigma p
      cplx<T> hv = hx[o + g];
      hv.x += a * (av.x + sg * pv.x);
      hv.y += a * (av.y + sg * pv.y);
      hx[o + g] = hv;
    }
    const double q = (double)rv.x * rv.x + (double)rv.y * rv.y;
    rr += q;
    rz += q * (double)((T)1 / (kin[g] + ps));
  }
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) prr[(size_t)gb * nch + ch] = rr;
  rz = block_sum(rz, red);
  if (threadIdx.x == 0) prz[(size_t)gb * nch + ch] = rz;
}

__global__ void k_bpcg_beta(int nbt, int nch, const double* __restrict__ prr, const double* __restrict__ prz,
                            const double* __restrict__ r0n, double tol, double* __restrict__ rz,
                            int* __restrict__ active, double* __restrict__ beta, int* __restrict__ still) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbt) return;
  if (!active[b]) {
    still[b] = 0;
    beta[b] = 0.0;
    return;
  }
  double q = 0.0, a = 0.0;
  for (int ch = 0; ch < nch; ++ch) {
    q += prr[(size_t)b * nch + ch];
    a += prz[(size_t)b * nch + ch];
  }
  const int s = sqrt(q) > tol * r0n[b] ? 1 : 0;
  beta[b] = s ? a / rz[b] : 0.0;
  if (s) rz[b] = a;
  still[b] = s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bpcg_pupdate(BandMap bm, cplx<T>* __restrict__ p, const cplx<T>* __restrict__ r,
                                                      const double* __restrict__ pshift, const double* __restrict__ beta,
                                                      int* __restrict__ still, int* __restrict__ active) {
  const int gb = blockIdx.y, ch = blockIdx.x;
  const int s = still[gb];
  if (ch == 0 && threadIdx.x == 0) active[gb] = s;  // active of the next step (this band's CTAs only read s)
  if (!s) return;
  const int pi = bm.prob[gb];
  const ProbDev& P = bm.probs[pi];
  const int npw = P.npw;
  const size_t o = P.off + (size_t)bm.row[gb] * npw;
  const T* kin = pd_kin<T>(P);
  const T ps = (T)pshift[pi];
  const T bt = (T)beta[gb];
  const int g0 = ch * kBChunk, g1 = min(npw, g0 + kBChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const T m = (T)1 / (kin[g] + ps);
    const cplx<T> rv = r[o + g], pv = p[o + g];
    p[o + g] = mk<T>(m * rv.x + bt * pv.x, m * rv.y + bt * pv.y);
  }
}

// rhs = T((eps_b - sigma_p) psi64), x = psi_T (Algorithm 1 source problems, started at psi)
// rhs = (eps - sigma) psi, x0 = psi, and (H - sigma) x0 = H psi - sigma psi from the H psi each context
// keeps with its orbitals (the last Rayleigh-Ritz step's), so the solves need no first H application
template <typename T>
__global__ void k_brhs(BandMap bm, const double2* __restrict__ psi64, const double2* __restrict__ hpsi64,
                       const double* __restrict__ eps, const double* __restrict__ sigma, cplx<T>* __restrict__ rhs,
                       cplx<T>* __restrict__ x, cplx<T>* __restrict__ ax, cplx<T>* __restrict__ hx) {
  const int gb = blockIdx.y;
  const int pi = bm.prob[gb];
  const ProbDev& P = bm.probs[pi];
  const int npw = P.npw;
  const size_t o = P.off + (size_t)bm.row[gb] * npw;
  const double sg = sigma[pi], f = eps[gb] - sg;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
    const double2 v = psi64[o + g], h = hpsi64[o + g];
    rhs[o + g] = mk<T>((T)(f * v.x), (T)(f * v.y));
    x[o + g] = mk<T>((T)v.x, (T)v.y);
    ax[o + g] = mk<T>((T)(h.x - sg * v.x), (T)(h.y - sg * v.y));
    if (hx) hx[o + g] = mk<T>((T)h.x, (T)h.y);
  }
}

// ------------------------------------------------------------------------------------------------
// projection step per problem
// ------------------------------------------------------------------------------------------------
// part[p][s] (64 x 64) = sum over K slice s of conj(A_m) B_n, m, n < nb_p; CARRY as in k_gemm_cn
template <typename T, bool CARRY>
__global__ void __launch_bounds__(256) k_bgram(const ProbDev* __restrict__ probs, int nslice,
                                               const cplx<T>* __restrict__ A, const cplx<T>* __restrict__ B,
                                               double2* __restrict__ part) {
  constexpr int R = 4, TILE = 64;
  const int s = blockIdx.x, pi = blockIdx.y;
  const ProbDev& P = probs[pi];
  const int nb = P.nb, npw = P.npw;
  const int k0 = s * kBSlice, k1 = min(npw, k0 + kBSlice);
  double2* out = part + ((size_t)pi * nslice + s) * TILE * TILE;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  if (k0 >= k1) {
    for (int i = tid; i < TILE * TILE; i += blockDim.x) out[i] = make_double2(0.0, 0.0);
    return;
  }
  __shared__ cplx<T> As[16][TILE + 1], Bs[16][TILE + 1];
  const cplx<T>* a = A + P.off;
  const cplx<T>* bb = B + P.off;
  cplx<T> acc[R][R];
  double2 cr[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      acc[i][j] = mk<T>(0, 0);
      cr[i][j] = make_double2(0.0, 0.0);
    }
  for (int kk = k0; kk < k1; kk += 16) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int i = tid + 256 * t;
      const int r = i >> 4, kx = i & 15, gk = kk + kx;
      As[kx][r] = (r < nb && gk < k1) ? cconj(a[(size_t)r * npw + gk]) : mk<T>(0, 0);
      Bs[kx][r] = (r < nb && gk < k1) ? bb[(size_t)r * npw + gk] : mk<T>(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kx = 0; kx < 16; ++kx) {
      cplx<T> av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        av[i] = As[kx][ty + 16 * i];
        bv[i] = Bs[kx][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          acc[i][j].x = fma(av[i].x, bv[j].x, acc[i][j].x);
          acc[i][j].x = fma(-av[i].y, bv[j].y, acc[i][j].x);
          acc[i][j].y = fma(av[i].x, bv[j].y, acc[i][j].y);
          acc[i][j].y = fma(av[i].y, bv[j].x, acc[i][j].y);
        }
    }
    if (CARRY) {
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          cr[i][j].x += (double)acc[i][j].x;
          cr[i][j].y += (double)acc[i][j].y;
          acc[i][j] = mk<T>(0, 0);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int m = ty + 16 * i, n = tx + 16 * j;
      out[m * TILE + n] = CARRY ? cr[i][j] : make_double2((double)acc[i][j].x, (double)acc[i][j].y);
    }
}

// S_p = sum_s part[p][s] (fixed order); hermitian: S <- (S + S^H) / 2
__global__ void k_bgram_reduce(const ProbDev* __restrict__ probs, int nslice, const double2* __restrict__ part,
                               double2* __restrict__ S, int hermitize) {
  const int pi = blockIdx.x;
  const int nb = probs[pi].nb;
  double2* Sp = S + (size_t)pi * kBMaxBands * kBMaxBands;
  const double2* pp = part + (size_t)pi * nslice * 64 * 64;
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
    const int m = i / nb, n = i - m * nb;
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    for (int s = 0; s < nslice; ++s) {
      a = cadd(a, pp[(size_t)s * 4096 + m * 64 + n]);
      if (hermitize) b = cadd(b, pp[(size_t)s * 4096 + n * 64 + m]);
    }
    Sp[m * kBMaxBands + n] = hermitize ? make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y)) : a;
  }
}

// Cholesky S = L L^H and G = conj(L)^{-1} (lower), one CTA per problem; info[p] = 1 if S is not positive
__global__ void __launch_bounds__(256) k_bchol(const ProbDev* __restrict__ probs, int ldm,
                                               const double2* __restrict__ S, double2* __restrict__ G,
                                               int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Lm = reinterpret_cast<double2*>(smem_raw);  // ldm x ldm, ldm = largest n_bands + 1
  __shared__ int s_bad;
  const int pi = blockIdx.x, n = probs[pi].nb;
#define L(i, j) Lm[(i) * ldm + (j)]
  const double2* Sp = S + (size_t)pi * kBMaxBands * kBMaxBands;
  double2* Gp = G + (size_t)pi * kBMaxBands * kBMaxBands;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) L(i / n, i % n) = Sp[(i / n) * kBMaxBands + (i % n)];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = L(j, j).x;
      if (!(d > 0.0) || !isfinite(d)) {
        s_bad = 1;
        L(j, j) = make_double2(1.0, 0.0);
      } else {
        L(j, j) = make_double2(sqrt(d), 0.0);
      }
    }
    __syncthreads();
    const double inv = 1.0 / L(j, j).x;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) L(i, j) = cscale(L(i, j), inv);
    __syncthreads();
    const int m = n - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {  // trailing update, lower part
      const int i = j + 1 + t / m, k = j + 1 + t % m;
      if (k <= i) L(i, k) = csub(L(i, k), cmul(L(i, j), cconj(L(k, j))));
    }
    __syncthreads();
  }
  // column c of L^{-1} by forward substitution, thread per column; G = conj(L^{-1})
  if (threadIdx.x < n) {
    const int c = threadIdx.x;
    for (int i = 0; i < n; ++i) {
      double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int k = c; k < i; ++k) s = csub(s, cmul(L(i, k), Gp[k * kBMaxBands + c]));
      Gp[i * kBMaxBands + c] = i < c ? make_double2(0.0, 0.0) : cscale(s, 1.0 / L(i, i).x);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    double2& g = Gp[(i / n) * kBMaxBands + (i % n)];
    g = cconj(g);
  }
  if (threadIdx.x == 0) info[pi] = s_bad;
}
#undef L

// Hermitian eigensolver (cyclic Jacobi, parallel round-robin ordering), one CTA per problem:
// w ascending, V[i][j] = component i of eigenvector j. Stops when the off-diagonal Frobenius norm is below
// 1e-13 of the whole; info[p] |= 2 if it is still above 1e-10 after 40 sweeps.
__global__ void __launch_bounds__(256) k_bjacobi(const ProbDev* __restrict__ probs, int ldm,
                                                 const double2* __restrict__ Ain, double* __restrict__ w,
                                                 double2* __restrict__ Vout, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Am = reinterpret_cast<double2*>(smem_raw);  // ldm x ldm each, ldm = largest n_bands + 1
  double2* Vm = Am + ldm * ldm;
#define A(i, j) Am[(i) * ldm + (j)]
#define V(i, j) Vm[(i) * ldm + (j)]
  __shared__ int pos[kBMaxBands];
  __shared__ double rc[kBMaxBands / 2], rs[kBMaxBands / 2];
  __shared__ double2 rph[kBMaxBands / 2];
  __shared__ int rp[kBMaxBands / 2], rq[kBMaxBands / 2];
  __shared__ double red[32];
  __shared__ double s_off, s_tot;
  __shared__ int perm[kBMaxBands];
  const int pi = blockIdx.x, n = probs[pi].nb;
  const double2* Ap = Ain + (size_t)pi * kBMaxBands * kBMaxBands;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i % n;
    A(r, c) = Ap[r * kBMaxBands + c];
    V(r, c) = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  JacobiScratch sc{pos, rc, rs, rph, rp, rq, red, &s_off, &s_tot};
  const int converged = jacobi_herm(n, ldm, Am, Vm, sc);
  // ascending order (ties by index)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = A(i, i).x;
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double b = A(j, j).x;
      r += (b < a) || (b == a && j < i);
    }
    perm[r] = i;
  }
  __syncthreads();
  double* wp = w + (size_t)probs[pi].band0;
  double2* Vp = Vout + (size_t)pi * kBMaxBands * kBMaxBands;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    Vp[i * kBMaxBands + j] = V(i, perm[j]);
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) wp[j] = A(perm[j], perm[j]).x;
  if (threadIdx.x == 0 && !converged) atomicOr(&info[pi], 2);
}
#undef A
#undef V

// Y[m] = sum_k W(k, m) X[k] per problem (rows of the problem's nb bands); W(k, m) = W[k][m] or W[m][k]
template <typename T>
__global__ void __launch_bounds__(256) k_bwx(const ProbDev* __restrict__ probs, const double2* __restrict__ W, int wt,
                                             const cplx<T>* __restrict__ X, cplx<T>* __restrict__ Y) {
  constexpr int MB = 32;
  __shared__ cplx<T> Ws[kBMaxBands][MB];
  const int pi = blockIdx.y;
  const ProbDev& P = probs[pi];
  const int nb = P.nb, npw = P.npw;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const double2* Wp = W + (size_t)pi * kBMaxBands * kBMaxBands;
  const cplx<T>* x = X + P.off;
  cplx<T>* y = Y + P.off;
  for (int m0 = 0; m0 < nb; m0 += MB) {
    const int mb = min(MB, nb - m0);
    __syncthreads();
    for (int i = threadIdx.x; i < nb * MB; i += blockDim.x) {
      const int k = i / MB, mm = i % MB;
      double2 v = make_double2(0.0, 0.0);
      if (mm < mb) v = wt ? Wp[(m0 + mm) * kBMaxBands + k] : Wp[k * kBMaxBands + m0 + mm];
      Ws[k][mm] = mk<T>((T)v.x, (T)v.y);
    }
    __syncthreads();
    if (g >= npw) continue;
    cplx<T> acc[MB];
#pragma unroll
    for (int mm = 0; mm < MB; ++mm) acc[mm] = mk<T>(0, 0);
    for (int k = 0; k < nb; ++k) {
      const cplx<T> xv = x[(size_t)k * npw + g];
#pragma unroll
      for (int mm = 0; mm < MB; ++mm) acc[mm] = cadd(acc[mm], cmul(Ws[k][mm], xv));
    }
    for (int mm = 0; mm < mb; ++mm) y[(size_t)(m0 + mm) * npw + g] = acc[mm];
  }
}

// ||hpsi_b - eps_b psi_b|| per flat band (FP64 arrays)
__global__ void k_bresid(BandMap bm, const double2* __restrict__ psi, const double2* __restrict__ hpsi,
                         const double* __restrict__ eps, double* __restrict__ res) {
  __shared__ double red[32];
  const int gb = blockIdx.x;
  const ProbDev& P = bm.probs[bm.prob[gb]];
  const int npw = P.npw;
  const size_t o = P.off + (size_t)bm.row[gb] * npw;
  const double e = eps[gb];
  double acc = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 p = psi[o + g], h = hpsi[o + g];
    const double re = h.x - e * p.x, im = h.y - e * p.y;
    acc += re * re + im * im;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) res[gb] = sqrt(acc);
}

template <typename TS, typename TD>
__global__ void k_bconvert(size_t n, const cplx<TS>* __restrict__ s, cplx<TD>* __restrict__ d) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = mk<TD>((TD)s[i].x, (TD)s[i].y);
}

}  // namespace paro

using namespace paro;

// ================================================================================================
// the batch object and its C ABI
// ================================================================================================
struct paro_batch {
  std::vector<paro_ctx*> ctxs;
  std::vector<std::pair<int, int>> pk;  // (context, k-point) of each problem
  Ctx* lead = nullptr;
  cudaStream_t st = nullptr;  // the contexts' stream (H psi calls, set-up)
  cudaStream_t gst = nullptr; // the batch's own stream: the captured step runs here
  cudaEvent_t ev = nullptr;
  bool f64 = true;
  int nprob = 0, nbt = 0, nitems = 0, nch = 1, nslice = 1;
  size_t nelem = 0;      // complex elements of one batch vector
  size_t smem = 0;       // bytes of the fused kernel's dynamic shared memory
  int threads = 1, grid = 152;  // autotuner's choice: launches per H psi (1 cooperative or 3) and grid
  void *sbuf = nullptr, *dpbuf = nullptr;  // stick buffers and scaled projections of the H psi phases
  int2 *d_u1 = nullptr, *d_u2 = nullptr, *d_u3 = nullptr;
  int n1 = 0, n2 = 0, n3 = 0;
  int sg = 64, ppt = 4096;         // work-unit shapes (autotuned)
  std::vector<int2> h_items;       // (problem, band) of every item, largest problems first
  std::vector<std::array<double, 5>> tuning;  // launches per apply, grid, sg, ppt, ms per apply
  unsigned* d_bar = nullptr;  // grid barrier (count, generation) and its time-out flag
  int ldm = 1;                     // largest n_bands + 1 (leading dimension of the per-problem matrices in
  size_t small_smem = 0;           // shared memory); bytes of the Jacobi kernel's two ldm x ldm matrices
  std::vector<ProbDev> hprob;
  ProbDev* d_prob = nullptr;
  int2* d_items = nullptr;
  int *d_bprob = nullptr, *d_brow = nullptr;
  // vectors (T = double or float by precision; FP64 copies always)
  void *x = nullptr, *r = nullptr, *p = nullptr, *ap = nullptr, *rhs = nullptr, *y = nullptr, *hy = nullptr;
  double2 *psi64 = nullptr, *hpsi64 = nullptr;
  double *prz = nullptr, *prr = nullptr, *rz = nullptr, *r0n = nullptr, *alpha = nullptr, *beta = nullptr;
  int *active = nullptr, *still = nullptr, *flags = nullptr;  // flags[0] = PCG breakdown, then per problem info
  double2 *part = nullptr, *S = nullptr, *G = nullptr;
  double *eps = nullptr, *res = nullptr, *sigma = nullptr, *pshift = nullptr;
  double* h_stage = nullptr;  // pinned: eps then res then sigma then pshift
  int* h_flags = nullptr;     // pinned
  cudaGraphExec_t exec = nullptr;   // the step that carries H x through the solves (H Y = G H X)
  cudaGraphExec_t exec2 = nullptr;  // the step that applies H to the Rayleigh-Ritz basis directly
  long long graph_kernels2 = 0;
  int hx_recur = 0;                 // carried steps since the last direct one
  void* hx = nullptr;
  double g_tol = -1.0;
  int g_maxit = -1;
  long long graph_kernels = 0;
  std::string err;
};

namespace {

int berr(paro_batch* b, int code, const std::string& msg) {
  b->err = msg;
  if (b->lead) b->lead->err = msg;
  return code;
}

#define BCU(b, call)                                                                          \
  do {                                                                                        \
    cudaError_t e__ = (call);                                                                 \
    if (e__ != cudaSuccess) return berr((b), PARO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
  } while (0)
#define BLAUNCH(b, what)                                                                      \
  do {                                                                                        \
    cudaError_t e__ = cudaGetLastError();                                                     \
    if (e__ != cudaSuccess) return berr((b), PARO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e__)); \
    ++(b)->graph_kernels;                                                                     \
  } while (0)

BandMap bandmap(const paro_batch* b) { return BandMap{b->d_bprob, b->d_brow, b->d_prob}; }

// One H psi over every item: mode 0 = one cooperative launch of the three phases, mode 1 = three launches.
template <typename T>
int launch_fused(paro_batch* b, cudaStream_t s, const cplx<T>* X, cplx<T>* Y, const int* active, int shifted,
                 int mode, int grid) {
  const HpsiLists L{b->d_u1, b->n1, b->d_u2, b->n2, b->d_u3, b->n3, b->sg, b->ppt};
  cplx<T>* S = static_cast<cplx<T>*>(b->sbuf);
  cplx<T>* DP = static_cast<cplx<T>*>(b->dpbuf);
  int* err = reinterpret_cast<int*>(b->d_bar + 2);
  if (mode == 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BCU(b, cudaLaunchKernelEx(&cfg, k_hpsi_batch<T, 0>, (const ProbDev*)b->d_prob, (const int2*)b->d_items, L, X, Y, S,
                              DP, active, (const double*)b->sigma, shifted, b->d_bar, err));
    ++b->graph_kernels;
    return PARO_OK;
  }
  k_hpsi_batch<T, 1><<<std::min(grid, b->n1), 256, b->smem, s>>>(b->d_prob, b->d_items, L, X, Y, S, DP, active,
                                                                  b->sigma, shifted, b->d_bar, err);
  BLAUNCH(b, "k_hpsi_batch<1>");
  k_hpsi_batch<T, 2><<<std::min(grid, b->n2), 256, b->smem, s>>>(b->d_prob, b->d_items, L, X, Y, S, DP, active,
                                                                  b->sigma, shifted, b->d_bar, err);
  BLAUNCH(b, "k_hpsi_batch<2>");
  k_hpsi_batch<T, 3><<<std::min(grid, b->n3), 256, b->smem, s>>>(b->d_prob, b->d_items, L, X, Y, S, DP, active,
                                                                  b->sigma, shifted, b->d_bar, err);
  BLAUNCH(b, "k_hpsi_batch<3>");
  return PARO_OK;
}

// the whole ParO step (Algorithm 1) for every problem, enqueued without any host wait
template <typename T>
int enqueue_step(paro_batch* b, double tol, int maxit, bool carry_hx) {
  cplx<T>* x = static_cast<cplx<T>*>(b->x);
  cplx<T>* r = static_cast<cplx<T>*>(b->r);
  cplx<T>* p = static_cast<cplx<T>*>(b->p);
  cplx<T>* ap = static_cast<cplx<T>*>(b->ap);
  cplx<T>* rhs = static_cast<cplx<T>*>(b->rhs);
  cplx<T>* y = static_cast<cplx<T>*>(b->y);
  cplx<T>* hy = static_cast<cplx<T>*>(b->hy);
  const BandMap bm = bandmap(b);
  cudaStream_t s_ = b->gst;
  const dim3 gv(b->nch, b->nbt);
  const int tb = (b->nbt + 127) / 128;
  int st;
  // gather the current orbitals (FP64) of every problem
  for (int i = 0; i < b->nprob; ++i) {
    const ProbDev& P = b->hprob[i];
    const Basis& B = unwrap(b->ctxs[b->pk[i].first])->bases[b->pk[i].second];
    BCU(b, cudaMemcpyAsync(b->psi64 + P.off, B.d_psi, (size_t)P.nb * P.npw * sizeof(double2),
                           cudaMemcpyDeviceToDevice, s_));
    BCU(b, cudaMemcpyAsync(b->hpsi64 + P.off, B.d_hpsi, (size_t)P.nb * P.npw * sizeof(double2),
                           cudaMemcpyDeviceToDevice, s_));
  }
  BCU(b, cudaMemsetAsync(b->flags, 0, (size_t)(1 + b->nprob) * sizeof(int), s_));
  // step 3: (H - sigma) x = (eps - sigma) psi, x0 = psi
  cplx<T>* hx = carry_hx ? static_cast<cplx<T>*>(b->hx) : nullptr;
  k_brhs<T><<<dim3(4, b->nbt), 256, 0, s_>>>(bm, b->psi64, b->hpsi64, b->eps, b->sigma, rhs, x, ap, hx);
  BLAUNCH(b, "k_brhs");
  k_bpcg_init<T><<<gv, 256, 0, s_>>>(bm, b->nch, rhs, ap, r, p, b->pshift, b->prz, b->prr);
  BLAUNCH(b, "k_bpcg_init");
  k_bpcg_band_init<<<tb, 128, 0, s_>>>(b->nbt, b->nch, b->prz, b->prr, b->rz, b->r0n, b->active);
  BLAUNCH(b, "k_bpcg_band_init");
  for (int it = 0; it < maxit; ++it) {
    if ((st = launch_fused<T>(b, s_, p, ap, b->active, 1, b->threads == 1 ? 0 : 1, b->grid))) return st;
    k_bpcg_dot<T><<<gv, 256, 0, s_>>>(bm, b->nch, p, ap, b->active, b->prz);
    BLAUNCH(b, "k_bpcg_dot");
    k_bpcg_alpha<<<tb, 128, 0, s_>>>(b->nbt, b->nch, b->prz, b->rz, b->active, b->alpha, b->flags);
    BLAUNCH(b, "k_bpcg_alpha");
    k_bpcg_update<T><<<gv, 256, 0, s_>>>(bm, b->nch, x, r, p, ap, b->pshift, b->alpha, b->active, b->prr,
                                             b->prz, hx, b->sigma);
    BLAUNCH(b, "k_bpcg_update");
    k_bpcg_beta<<<tb, 128, 0, s_>>>(b->nbt, b->nch, b->prr, b->prz, b->r0n, tol, b->rz, b->active, b->beta,
                                       b->still);
    BLAUNCH(b, "k_bpcg_beta");
    k_bpcg_pupdate<T><<<gv, 256, 0, s_>>>(bm, p, r, b->pshift, b->beta, b->still, b->active);
    BLAUNCH(b, "k_bpcg_pupdate");
  }
  // step 4: Cholesky-orthonormalise X, Rayleigh-Ritz in its span
  const bool carry = sizeof(T) == 4;
  const dim3 gg(b->nslice, b->nprob);
  if (carry)
    k_bgram<T, true><<<gg, 256, 0, s_>>>(b->d_prob, b->nslice, x, x, b->part);
  else
    k_bgram<T, false><<<gg, 256, 0, s_>>>(b->d_prob, b->nslice, x, x, b->part);
  BLAUNCH(b, "k_bgram");
  k_bgram_reduce<<<b->nprob, 256, 0, s_>>>(b->d_prob, b->nslice, b->part, b->S, 1);
  BLAUNCH(b, "k_bgram_reduce");
  k_bchol<<<b->nprob, 256, b->small_smem / 2, s_>>>(b->d_prob, b->ldm, b->S, b->G, b->flags + 1);
  BLAUNCH(b, "k_bchol");
  const dim3 gw((b->nch * kBChunk + 255) / 256, b->nprob);
  k_bwx<T><<<gw, 256, 0, s_>>>(b->d_prob, b->G, 1, x, y);
  BLAUNCH(b, "k_bwx");
  if (carry_hx) {  // H Y = G (H X): the potential is fixed within the step
    k_bwx<T><<<gw, 256, 0, s_>>>(b->d_prob, b->G, 1, hx, hy);
    BLAUNCH(b, "k_bwx");
  } else if ((st = launch_fused<T>(b, s_, y, hy, nullptr, 0, b->threads == 1 ? 0 : 1, b->grid))) {
    return st;
  }
  if (carry)
    k_bgram<T, true><<<gg, 256, 0, s_>>>(b->d_prob, b->nslice, y, hy, b->part);
  else
    k_bgram<T, false><<<gg, 256, 0, s_>>>(b->d_prob, b->nslice, y, hy, b->part);
  BLAUNCH(b, "k_bgram");
  k_bgram_reduce<<<b->nprob, 256, 0, s_>>>(b->d_prob, b->nslice, b->part, b->S, 1);
  BLAUNCH(b, "k_bgram_reduce");
  k_bjacobi<<<b->nprob, 256, b->small_smem, s_>>>(b->d_prob, b->ldm, b->S, b->eps, b->G, b->flags + 1);
  BLAUNCH(b, "k_bjacobi");
  k_bwx<T><<<gw, 256, 0, s_>>>(b->d_prob, b->G, 0, y, x);   // psi
  BLAUNCH(b, "k_bwx");
  k_bwx<T><<<gw, 256, 0, s_>>>(b->d_prob, b->G, 0, hy, r);  // H psi
  BLAUNCH(b, "k_bwx");
  if (sizeof(T) == 4) {
    k_bconvert<T, double><<<1024, 256, 0, s_>>>(b->nelem, x, b->psi64);
    BLAUNCH(b, "k_bconvert");
    k_bconvert<T, double><<<1024, 256, 0, s_>>>(b->nelem, r, b->hpsi64);
    BLAUNCH(b, "k_bconvert");
  } else {
    BCU(b, cudaMemcpyAsync(b->psi64, x, b->nelem * sizeof(double2), cudaMemcpyDeviceToDevice, s_));
    BCU(b, cudaMemcpyAsync(b->hpsi64, r, b->nelem * sizeof(double2), cudaMemcpyDeviceToDevice, s_));
  }
  k_bresid<<<b->nbt, 256, 0, s_>>>(bm, b->psi64, b->hpsi64, b->eps, b->res);
  BLAUNCH(b, "k_bresid");
  // scatter the new orbitals back to their contexts; eigenvalues, residuals and flags to pinned host memory
  for (int i = 0; i < b->nprob; ++i) {
    const ProbDev& P = b->hprob[i];
    Basis& B = unwrap(b->ctxs[b->pk[i].first])->bases[b->pk[i].second];
    const size_t n = (size_t)P.nb * P.npw;
    BCU(b, cudaMemcpyAsync(B.d_psi, b->psi64 + P.off, n * sizeof(double2), cudaMemcpyDeviceToDevice, s_));
    BCU(b, cudaMemcpyAsync(B.d_hpsi, b->hpsi64 + P.off, n * sizeof(double2), cudaMemcpyDeviceToDevice, s_));
    if (sizeof(T) == 4) {
      BCU(b, cudaMemcpyAsync(B.d_psi32, static_cast<float2*>(b->x) + P.off, n * sizeof(float2),
                             cudaMemcpyDeviceToDevice, s_));
      BCU(b, cudaMemcpyAsync(B.d_hpsi32, static_cast<float2*>(b->r) + P.off, n * sizeof(float2),
                             cudaMemcpyDeviceToDevice, s_));
    }
  }
  BCU(b, cudaMemcpyAsync(b->h_stage, b->eps, (size_t)b->nbt * sizeof(double), cudaMemcpyDeviceToHost, s_));
  BCU(b, cudaMemcpyAsync(b->h_stage + b->nbt, b->res, (size_t)b->nbt * sizeof(double), cudaMemcpyDeviceToHost,
                         s_));
  BCU(b, cudaMemcpyAsync(b->h_flags, b->flags, (size_t)(1 + b->nprob) * sizeof(int), cudaMemcpyDeviceToHost, s_));
  return PARO_OK;
}

// The three work lists for unit shapes (sg, ppt) on the device, and the shared memory they need (bytes).
// Returns PARO_ERR_ARG (nothing changed) when a unit does not fit one CTA's shared memory.
int build_lists(paro_batch* b, int sg, int ppt) {
  const size_t es = b->f64 ? sizeof(double2) : sizeof(float2);
  size_t max_el = 0;
  for (const ProbDev& P : b->hprob) max_el = std::max(max_el, unit_elems(P, sg, ppt));
  if (max_el * es > 227 * 1024) return PARO_ERR_ARG;
  std::vector<int2> u1, u2, u3;
  for (int it = 0; it < (int)b->h_items.size(); ++it) {
    const ProbDev& P = b->hprob[b->h_items[it].x];
    const int ng = (P.ncol + sg - 1) / sg;
    if (P.nproj > 0) u1.push_back(make_int2(it, -1));
    for (int g = 0; g < ng; ++g) {
      u1.push_back(make_int2(it, g));
      u3.push_back(make_int2(it, g));
    }
    for (int z = 0; z < P.N3; z += planes_per_unit(P.N1, P.N2, ppt)) u2.push_back(make_int2(it, z));
  }
  BCU(b, cudaStreamSynchronize(b->st));
  int2** dst[3] = {&b->d_u1, &b->d_u2, &b->d_u3};
  const std::vector<int2>* src[3] = {&u1, &u2, &u3};
  for (int i = 0; i < 3; ++i) {
    if (*dst[i]) cudaFree(*dst[i]);
    *dst[i] = nullptr;
    BCU(b, cudaMalloc(dst[i], std::max<size_t>(src[i]->size(), 1) * sizeof(int2)));
    BCU(b, cudaMemcpy(*dst[i], src[i]->data(), src[i]->size() * sizeof(int2), cudaMemcpyHostToDevice));
  }
  b->n1 = (int)u1.size();
  b->n2 = (int)u2.size();
  b->n3 = (int)u3.size();
  b->sg = sg;
  b->ppt = ppt;
  b->smem = max_el * es;
  return PARO_OK;
}

template <typename T>
int autotune(paro_batch* b) {
  int dev = 0, sms = 0;
  BCU(b, cudaGetDevice(&dev));
  BCU(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BCU(b, cudaFuncSetAttribute(k_bjacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->small_smem));
  BCU(b, cudaFuncSetAttribute(k_bchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->small_smem));
  cplx<T>* X = static_cast<cplx<T>*>(b->p);
  cplx<T>* Y = static_cast<cplx<T>*>(b->ap);
  BCU(b, cudaMemsetAsync(X, 0, b->nelem * sizeof(cplx<T>), b->st));
  cudaEvent_t e0, e1;
  BCU(b, cudaEventCreate(&e0));
  BCU(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_sg = 64, best_ppt = 4096;
  b->tuning.clear();
  // unit shapes x launch form (one cooperative launch, or one launch per phase) x grid (CTAs per SM)
  for (int sg : {32, 64, 128})
    for (int ppt : {2048, 4096, 8192}) {
      if (build_lists(b, sg, ppt) != PARO_OK) continue;  // the unit does not fit shared memory
      for (int ph = 0; ph < 4; ++ph) {
        const void* fn = ph == 0 ? (const void*)k_hpsi_batch<T, 0>
                         : ph == 1 ? (const void*)k_hpsi_batch<T, 1>
                         : ph == 2 ? (const void*)k_hpsi_batch<T, 2> : (const void*)k_hpsi_batch<T, 3>;
        BCU(b, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
      }
      for (int mode : {0, 1}) {
        int per_sm = 0;
        if (mode == 0)
          BCU(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hpsi_batch<T, 0>, 256, b->smem));
        else
          BCU(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hpsi_batch<T, 2>, 256, b->smem));
        for (int mult : {1, 2, 4, 8}) {  // mode 0: co-resident CTAs only
          if (mult > per_sm) break;
          const int grid = mult * sms;
          int st;
          if ((st = launch_fused<T>(b, b->st, X, Y, nullptr, 0, mode, grid))) return st;
          BCU(b, cudaEventRecord(e0, b->st));
          for (int rep = 0; rep < 3; ++rep)
            if ((st = launch_fused<T>(b, b->st, X, Y, nullptr, 0, mode, grid))) return st;
          BCU(b, cudaEventRecord(e1, b->st));
          BCU(b, cudaEventSynchronize(e1));
          float ms = 0.f;
          BCU(b, cudaEventElapsedTime(&ms, e0, e1));
          b->tuning.push_back({(double)(mode == 0 ? 1 : 3), (double)grid, (double)sg, (double)ppt, ms / 3.0});
          if (ms < best) {
            best = ms;
            b->threads = mode == 0 ? 1 : 3;  // launches per H psi
            b->grid = grid;
            best_sg = sg;
            best_ppt = ppt;
          }
        }
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best >= 1e30f) return berr(b, PARO_ERR_ARG, "batch: H psi kernel cannot be resident");
  int st = build_lists(b, best_sg, best_ppt);
  if (st) return berr(b, st, "batch: work lists");
  for (int ph = 0; ph < 4; ++ph) {
    const void* fn = ph == 0 ? (const void*)k_hpsi_batch<T, 0>
                     : ph == 1 ? (const void*)k_hpsi_batch<T, 1>
                     : ph == 2 ? (const void*)k_hpsi_batch<T, 2> : (const void*)k_hpsi_batch<T, 3>;
    BCU(b, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  }
  unsigned h[3] = {0, 0, 0};
  BCU(b, cudaMemcpy(h, b->d_bar, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[2]) return berr(b, PARO_ERR_TIMEOUT, "batch: grid barrier wait gave up");
  b->graph_kernels = 0;
  return PARO_OK;
}

void free_batch(paro_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->exec2) cudaGraphExecDestroy(b->exec2);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->gst) cudaStreamDestroy(b->gst);
  void* bufs[] = {b->d_prob, b->d_items, b->d_bprob, b->d_brow, b->x, b->r, b->p, b->ap, b->rhs, b->y, b->hy, b->hx,
                  b->sbuf, b->dpbuf, b->d_u1, b->d_u2, b->d_u3, b->d_bar,
                  b->psi64, b->hpsi64, b->prz, b->prr, b->rz, b->r0n, b->alpha, b->beta, b->active, b->still,
                  b->flags, b->part, b->S, b->G, b->eps, b->res, b->sigma, b->pshift};
  for (void* q : bufs)
    if (q) cudaFree(q);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  delete b;
}

int refresh_scalars(paro_batch* b) {
  // eigenvalues of the current orbitals and each problem's shift, from the contexts
  for (int i = 0; i < b->nprob; ++i) {
    Ctx& c = *unwrap(b->ctxs[b->pk[i].first]);
    if (veff_stats(&c)) return berr(b, PARO_ERR_CUDA, "batch: " + c.err);
    const Basis& B = c.bases[b->pk[i].second];
    if (!B.have_psi || (int)B.eps.size() < c.nb)
      return berr(b, PARO_ERR_STATE, "batch: every context needs orbitals (paro_set_orbitals) first");
    for (int j = 0; j < c.nb; ++j) b->h_stage[b->hprob[i].band0 + j] = B.eps[j];
    b->h_stage[2 * b->nbt + i] = c.sigma_k[b->pk[i].second];
    b->h_stage[2 * b->nbt + b->nprob + i] = c.vmean - c.sigma_k[b->pk[i].second];
  }
  BCU(b, cudaMemcpyAsync(b->eps, b->h_stage, b->nbt * sizeof(double), cudaMemcpyHostToDevice, b->gst));
  BCU(b, cudaMemcpyAsync(b->sigma, b->h_stage + 2 * b->nbt, b->nprob * sizeof(double), cudaMemcpyHostToDevice,
                         b->gst));
  BCU(b, cudaMemcpyAsync(b->pshift, b->h_stage + 2 * b->nbt + b->nprob, b->nprob * sizeof(double),
                         cudaMemcpyHostToDevice, b->gst));
  return PARO_OK;
}

}  // namespace

extern "C" {

int paro_batch_create(paro_batch** out, paro_ctx* const* ctxs, int n_ctx) {
  if (!out || !ctxs || n_ctx < 1) return PARO_ERR_ARG;
  *out = nullptr;
  paro_batch* b = new paro_batch;
  b->ctxs.assign(ctxs, ctxs + n_ctx);
  for (int i = 0; i < n_ctx; ++i)
    if (!ctxs[i]) {
      delete b;
      return PARO_ERR_ARG;
    }
  b->lead = unwrap(ctxs[0]);
  b->st = b->lead->stream;
  b->f64 = b->lead->prec == PARO_FP64;
  const size_t es = b->f64 ? sizeof(double2) : sizeof(float2);
  auto bail = [&](int code, const std::string& msg) {
    b->lead->err = msg;
    free_batch(b);
    return code;
  };
  size_t off = 0, max_el = 0, soff = 0, dpoff = 0;
  int band0 = 0, max_npw = 0;
  for (int ci = 0; ci < n_ctx; ++ci) {
    Ctx& c = *unwrap(ctxs[ci]);
    if ((c.prec == PARO_FP64) != b->f64) return bail(PARO_ERR_ARG, "batch: contexts differ in precision");
    if (!c.have_veff) return bail(PARO_ERR_STATE, "batch: every context needs a potential");
    if (c.nb > kBMaxBands) return bail(PARO_ERR_ARG, "batch: at most 64 bands per context");
    if (c.gamma_real) return bail(PARO_ERR_ARG, "batch: contexts in the real-wavefunction mode are not batched");
    if (c.stream != b->st) return bail(PARO_ERR_ARG, "batch: contexts must share one stream");
    for (int ik = 0; ik < c.nk; ++ik) {
      const Basis& B = c.bases[ik];
      ProbDev P = {};
      P.npw = B.npw;
      P.ncol = B.ncol;
      P.nxr = B.nxr;
      P.nb = c.nb;
      P.N1 = c.N[0];
      P.N2 = c.N[1];
      P.N3 = c.N[2];
      P.nproj = c.have_kb ? c.nproj : 0;
      P.off = (long long)off;
      P.band0 = band0;
      for (int a = 0; a < 3; ++a) {
        P.plan[a] = c.plan[a];
        P.tw64[a] = c.d_tw64[a];
        P.tw32[a] = c.d_tw32[a];
      }
      P.col_x = B.d_col_x;
      P.col_y = B.d_col_y;
      P.col_off = B.d_col_off;
      P.g_col = B.d_g_col;
      P.g_z = B.d_g_z;
      P.xrows = B.d_xrows;
      P.kin = B.d_kin;
      P.kin32 = B.d_kin32;
      P.vplane = c.d_vplane;
      P.vplane32 = c.d_vplane32;
      P.beta = B.d_beta;
      P.beta32 = B.d_beta32;
      P.dvec = c.d_dvec;
      P.soff = (long long)soff;
      P.dpoff = (long long)dpoff;
      soff += (size_t)c.nb * P.N3 * P.ncol;
      dpoff += (size_t)c.nb * P.nproj;
      max_el = std::max(max_el, unit_elems(P, 32, 2048));
      b->hprob.push_back(P);
      b->pk.push_back({ci, ik});
      off += (size_t)c.nb * B.npw;
      band0 += c.nb;
      max_npw = std::max(max_npw, B.npw);
    }
  }
  b->nprob = (int)b->hprob.size();
  b->nbt = band0;
  b->nelem = off;
  if (max_el * es > 227 * 1024)  // the smallest unit shapes (32 sticks, one plane)
    return bail(PARO_ERR_ARG, "batch: a plane does not fit one CTA's shared memory (" + std::to_string(max_el * es) +
                                  " bytes)");
  int max_nb = 1;
  for (const ProbDev& P : b->hprob) max_nb = std::max(max_nb, P.nb);
  b->ldm = max_nb + 1;
  b->small_smem = (size_t)2 * b->ldm * b->ldm * sizeof(double2);
  b->nch = (max_npw + kBChunk - 1) / kBChunk;
  b->nslice = (max_npw + kBSlice - 1) / kBSlice;
  // items, largest problems first (their FFT work ~ N1 N2 N3)
  std::vector<int> order(b->nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c2) {
    const ProbDev &A = b->hprob[a], &C = b->hprob[c2];
    return (long long)A.N1 * A.N2 * A.N3 > (long long)C.N1 * C.N2 * C.N3;
  });
  std::vector<int2> items;
  for (int pi : order)
    for (int j = 0; j < b->hprob[pi].nb; ++j) items.push_back(make_int2(pi, j));
  b->nitems = (int)items.size();
  b->h_items = items;
  std::vector<int> bprob(b->nbt), brow(b->nbt);
  for (int pi = 0; pi < b->nprob; ++pi)
    for (int j = 0; j < b->hprob[pi].nb; ++j) {
      bprob[b->hprob[pi].band0 + j] = pi;
      brow[b->hprob[pi].band0 + j] = j;
    }
  const size_t vb = b->nelem * es;
  const size_t mat = (size_t)b->nprob * kBMaxBands * kBMaxBands * sizeof(double2);
  cudaError_t e = cudaSuccess;
  auto al = [&](void** q, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(q, std::max<size_t>(n, 16));
  };
  al((void**)&b->d_prob, b->nprob * sizeof(ProbDev));
  al((void**)&b->d_items, items.size() * sizeof(int2));
  al((void**)&b->d_bprob, b->nbt * sizeof(int));
  al((void**)&b->d_brow, b->nbt * sizeof(int));
  for (void** q : {&b->x, &b->r, &b->p, &b->ap, &b->rhs, &b->y, &b->hy, &b->hx}) al(q, vb);
  al((void**)&b->psi64, b->nelem * sizeof(double2));
  al((void**)&b->hpsi64, b->nelem * sizeof(double2));
  al((void**)&b->prz, (size_t)b->nbt * b->nch * sizeof(double));
  al((void**)&b->prr, (size_t)b->nbt * b->nch * sizeof(double));
  for (double** q : {&b->rz, &b->r0n, &b->alpha, &b->beta, &b->eps, &b->res}) al((void**)q, b->nbt * sizeof(double));
  al((void**)&b->sigma, b->nprob * sizeof(double));
  al((void**)&b->pshift, b->nprob * sizeof(double));
  al((void**)&b->active, b->nbt * sizeof(int));
  al((void**)&b->still, b->nbt * sizeof(int));
  al((void**)&b->flags, (1 + b->nprob) * sizeof(int));
  al((void**)&b->part, (size_t)b->nprob * b->nslice * 4096 * sizeof(double2));
  al(&b->sbuf, soff * es);
  al(&b->dpbuf, std::max<size_t>(dpoff, 1) * es);
  al((void**)&b->d_bar, 4 * sizeof(unsigned));
  al((void**)&b->S, mat);
  al((void**)&b->G, mat);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gst, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_stage, (2 * (size_t)b->nbt + 2 * b->nprob) * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_flags, (1 + b->nprob) * sizeof(int));
  if (e != cudaSuccess) return bail(PARO_ERR_CUDA, std::string("batch allocation: ") + cudaGetErrorString(e));
  e = cudaMemcpy(b->d_prob, b->hprob.data(), b->nprob * sizeof(ProbDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_bprob, bprob.data(), b->nbt * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_brow, brow.data(), b->nbt * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, 4 * sizeof(unsigned));
  if (e != cudaSuccess) return bail(PARO_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  const int st = b->f64 ? autotune<double>(b) : autotune<float>(b);
  if (st) {
    const std::string msg = b->err;
    return bail(st, msg);
  }
  *out = b;
  return PARO_OK;
}

int paro_batch_apply_h(paro_batch* b, int dtype, const void* const* psi, void* const* hpsi) {
  if (!b || !psi || !hpsi) return PARO_ERR_ARG;
  if ((dtype == PARO_C64) != b->f64 || (dtype != PARO_C64 && dtype != PARO_C32))
    return berr(b, PARO_ERR_ARG, "paro_batch_apply_h: dtype must match the contexts' precision");
  const size_t es = b->f64 ? sizeof(double2) : sizeof(float2);
  for (int i = 0; i < b->nprob; ++i) {
    const ProbDev& P = b->hprob[i];
    if (!psi[i] || !hpsi[i]) return berr(b, PARO_ERR_ARG, "paro_batch_apply_h: null pointer");
    BCU(b, cudaMemcpyAsync(static_cast<char*>(b->p) + P.off * es, psi[i], (size_t)P.nb * P.npw * es,
                           cudaMemcpyDeviceToDevice, b->st));
  }
  const int mode = b->threads == 1 ? 0 : 1;
  int st = b->f64 ? launch_fused<double>(b, b->st, static_cast<const double2*>(b->p), static_cast<double2*>(b->ap),
                                         nullptr, 0, mode, b->grid)
                  : launch_fused<float>(b, b->st, static_cast<const float2*>(b->p), static_cast<float2*>(b->ap),
                                        nullptr, 0, mode, b->grid);
  if (st) return st;
  b->lead->launches += 1;
  for (int i = 0; i < b->nprob; ++i) {
    const ProbDev& P = b->hprob[i];
    BCU(b, cudaMemcpyAsync(hpsi[i], static_cast<char*>(b->ap) + P.off * es, (size_t)P.nb * P.npw * es,
                           cudaMemcpyDeviceToDevice, b->st));
  }
  return PARO_OK;
}

int paro_batch_step(paro_batch* b, double rel_tol, int max_it, double* max_resid_out) {
  if (!b || max_it < 0 || !(rel_tol >= 0)) return PARO_ERR_ARG;
  int st;
  // the batch reads each context's FP64 orbitals and H psi (it writes both precisions back)
  for (int i = 0; i < b->nprob; ++i) {
    Ctx& cx = *unwrap(b->ctxs[b->pk[i].first]);
    Basis& B = cx.bases[b->pk[i].second];
    if ((B.psi64_stale || B.hpsi64_stale) && fp64_current(&cx, B)) return berr(b, PARO_ERR_CUDA, "batch: " + cx.err);
    B.psi64_stale = B.hpsi64_stale = false;
  }
  BCU(b, cudaEventRecord(b->ev, b->st));  // work queued on the contexts' stream comes first
  BCU(b, cudaStreamWaitEvent(b->gst, b->ev, 0));
  if ((st = refresh_scalars(b))) return st;
  if (rel_tol != b->g_tol || max_it != b->g_maxit) {  // new parameters: both graphs are stale
    for (cudaGraphExec_t* e : {&b->exec, &b->exec2})
      if (*e) {
        cudaGraphExecDestroy(*e);
        *e = nullptr;
      }
    b->g_tol = rel_tol;
    b->g_maxit = max_it;
  }
  // eight steps carry H X through the solves, the ninth applies H to the Rayleigh-Ritz basis directly, so
  // the FP32 rounding of the carried H psi cannot accumulate
  const bool carry = b->hx_recur < 8;
  b->hx_recur = carry ? b->hx_recur + 1 : 0;
  for (int form = 0; form < 2; ++form) {  // both graphs at once, so no capture falls inside later steps
  const bool fcarry = form == 0;
  cudaGraphExec_t& exec = fcarry ? b->exec : b->exec2;
  long long& nk = fcarry ? b->graph_kernels : b->graph_kernels2;
  if (!exec) {
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaSuccess;
    for (int attempt = 0; attempt < 2; ++attempt) {
      BCU(b, cudaStreamBeginCapture(b->gst, cudaStreamCaptureModeThreadLocal));
      const long long k0 = b->graph_kernels;
      b->graph_kernels = 0;
      st = b->f64 ? enqueue_step<double>(b, rel_tol, max_it, fcarry)
                  : enqueue_step<float>(b, rel_tol, max_it, fcarry);
      nk = b->graph_kernels;
      if (!fcarry) b->graph_kernels = k0;
      ec = cudaStreamEndCapture(b->gst, &g);
      if (st == PARO_OK && ec == cudaSuccess) break;
      if (g) cudaGraphDestroy(g);
      g = nullptr;
      cudaGetLastError();
      if (b->threads != 1) break;
      b->threads = 3;  // capture the three-launch form of H psi instead of the cooperative one
    }
    if (st) return st;
    if (ec != cudaSuccess) return berr(b, PARO_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return berr(b, PARO_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  }
  }
  BCU(b, cudaGraphLaunch(carry ? b->exec : b->exec2, b->gst));
  BCU(b, cudaStreamSynchronize(b->gst));
  b->lead->launches += carry ? b->graph_kernels : b->graph_kernels2;
  unsigned hb[3] = {0, 0, 0};
  BCU(b, cudaMemcpy(hb, b->d_bar, sizeof(hb), cudaMemcpyDeviceToHost));
  if (hb[2]) return berr(b, PARO_ERR_TIMEOUT, "batch: grid barrier wait gave up");
  if (b->h_flags[0])
    return berr(b, PARO_ERR_BREAKDOWN, "batch PCG breakdown in band " + std::to_string(b->h_flags[0] - 1));
  double mx = 0.0;
  for (int i = 0; i < b->nprob; ++i) {
    if (b->h_flags[1 + i] & 1) return berr(b, PARO_ERR_BREAKDOWN, "batch: Gram matrix not positive definite");
    if (b->h_flags[1 + i] & 2) return berr(b, PARO_ERR_NOT_CONVERGED, "batch: Jacobi eigensolver did not converge");
    Ctx& c = *unwrap(b->ctxs[b->pk[i].first]);
    Basis& B = c.bases[b->pk[i].second];
    const int b0 = b->hprob[i].band0;
    B.eps.assign(b->h_stage + b0, b->h_stage + b0 + c.nb);
    B.res.assign(b->h_stage + b->nbt + b0, b->h_stage + b->nbt + b0 + c.nb);
    B.have_psi = true;
    for (int j = 0; j < c.nocc; ++j) mx = std::max(mx, B.res[j]);
  }
  if (max_resid_out) *max_resid_out = mx;
  return PARO_OK;
}

int paro_batch_info(const paro_batch* b, int* n_problems, int* n_items, int* launches_per_apply, int* grid,
                    long long* kernels_per_step) {
  if (!b) return PARO_ERR_ARG;
  if (n_problems) *n_problems = b->nprob;
  if (n_items) *n_items = b->nitems;
  if (launches_per_apply) *launches_per_apply = b->threads;
  if (grid) *grid = b->grid;
  if (kernels_per_step) *kernels_per_step = b->exec ? b->graph_kernels : 0;
  return PARO_OK;
}

int paro_batch_tuning(const paro_batch* b, int max_rows, int* n_rows, double* rows) {
  if (!b || !n_rows || max_rows < 0 || (max_rows > 0 && !rows)) return PARO_ERR_ARG;
  const int n = (int)b->tuning.size();
  *n_rows = n;
  for (int i = 0; i < n && i < max_rows; ++i)
    for (int j = 0; j < 5; ++j) rows[5 * i + j] = b->tuning[i][j];
  return PARO_OK;
}

void paro_batch_destroy(paro_batch* b) {
  if (b) free_batch(b);
}

}  // extern "C"
