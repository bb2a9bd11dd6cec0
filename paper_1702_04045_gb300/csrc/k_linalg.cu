// Dense complex linear algebra of the ParO projection step (Algorithm 1 step 4, Algorithm 2 step 4):
// Gram and Rayleigh-Ritz matrices (long-K "conj(A) B^T" GEMM, split over K with a fixed-order
// reduction), subspace rotations (short-K update GEMM), Cholesky orthonormalisation and the
// Hermitian eigensolver of the small Rayleigh-Ritz problem.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>
#include <cstdlib>

#include "paro_ctx.h"

namespace paro {

template <typename A, typename B> struct Promote { using t = double; };
template <> struct Promote<float, float> { using t = float; };

template <typename TO, typename TI> __device__ __forceinline__ cplx<TO> cvt(cplx<TI> v) {
  return mk<TO>((TO)v.x, (TO)v.y);
}

// ------------------------------------------------------------------------------------------------
// C = conj(A) B^T, (16 R) x (16 R) output tile per CTA (256 threads, R x R complex accumulators each,
// rows ty + 16 i and columns tx + 16 j), K split over gridDim.z into fixed slices of 16-wide steps.
// part[z][m][n] receives the slice sums (complex double). R is chosen per call to minimise padding.
// ACC = double: every product and sum in FP64. ACC = float: FP32 sums over the K slice, or with CARRY the
// 16 products of one K step are summed in FP32 and the step sums are added into an unevaluated pair
// hi + lo of FP32 values (error-free two-sum, Knuth; lo gathers the rounding error of every addition),
// so the FP32 rounding is that of a 16-term sum (the size of the rounding already in FP32 operands) and
// does not grow with K, without FP64 instructions in the loop (FP64 issues at 1/64 of the FP32 rate here).
// ------------------------------------------------------------------------------------------------
// K values per pipeline stage: 32 for FP32 operands (half the barriers per product of the 16-value stage),
// 16 for FP64 (the stage's shared memory doubles with the element size)
template <typename ACC> struct CnStepK { static constexpr int value = 32; };
template <> struct CnStepK<double> { static constexpr int value = 16; };

template <typename TA, typename TB, typename ACC, int R, bool CARRY>
__global__ void __launch_bounds__(256) k_gemm_cn(int M, int N, int K, int kslice, const cplx<TA>* __restrict__ A,
                                                 int lda, const cplx<TB>* __restrict__ B, int ldb,
                                                 double2* __restrict__ part, int herm) {
  constexpr int KS = CnStepK<ACC>::value;                          // K values per stage
  constexpr int TILE = 16 * R, LD = TILE + 1, STG = 2 * KS * LD;  // elements per stage (A then B)
  const int tm = blockIdx.y * TILE, tn = blockIdx.x * TILE;
  if (herm && tm > tn) return;
  const int k0 = blockIdx.z * kslice, k1 = min(K, k0 + kslice);
  extern __shared__ __align__(16) unsigned char cn_smem_raw[];
  cplx<ACC>* cn_smem = reinterpret_cast<cplx<ACC>*>(cn_smem_raw);  // two stages of As[16][LD], Bs[16][LD]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  constexpr bool kCarry = CARRY && sizeof(ACC) == 4;
  static_assert(sizeof(TA) == sizeof(ACC) && sizeof(TB) == sizeof(ACC), "operands are staged as stored");
  constexpr int EB = (int)sizeof(cplx<ACC>);
  // K step kk into stage buffer st by asynchronous copies (zero-filled outside); A is kept unconjugated
  auto stage = [&](int kk, int st) {
    cplx<ACC>* As = cn_smem + st * STG;
    cplx<ACC>* Bs = As + KS * LD;
#pragma unroll
    for (int t = 0; t < R * (KS / 16); ++t) {
      const int i = tid + 256 * t;
      const int r = i / KS, kx = i % KS, gk = kk + kx;
      const int gm = tm + r, gn = tn + r;
      const bool ia = gm < M && gk < k1, ib = gn < N && gk < k1;
      const cplx<TA>* sa = ia ? A + (size_t)gm * lda + gk : A;
      const cplx<TB>* sb = ib ? B + (size_t)gn * ldb + gk : B;
      if constexpr (EB == 8) {
        cp_async8(As + kx * LD + r, sa, ia ? 8 : 0);
        cp_async8(Bs + kx * LD + r, sb, ib ? 8 : 0);
      } else {
        cp_async16(As + kx * LD + r, sa, ia ? 16 : 0);
        cp_async16(Bs + kx * LD + r, sb, ib ? 16 : 0);
      }
    }
    cp_async_commit();
  };
  cplx<ACC> acc[R][R];
  float2 chi[R][R], clo[R][R];  // CARRY: running sum hi + lo
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      acc[i][j] = mk<ACC>(0, 0);
      chi[i][j] = clo[i][j] = make_float2(0.f, 0.f);
    }
  const int nk = k1 > k0 ? (k1 - k0 + KS - 1) / KS : 0;
  if (nk > 0) stage(k0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) {
      stage(k0 + KS * (kt + 1), (kt + 1) & 1);  // the other buffer: its readers passed the last barrier
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const cplx<ACC>* As = cn_smem + (kt & 1) * STG;
    const cplx<ACC>* Bs = As + KS * LD;
#pragma unroll
    for (int kh = 0; kh < KS / 16; ++kh) {  // 16 K values, then the carry
#pragma unroll 4
    for (int kx = 16 * kh; kx < 16 * kh + 16; ++kx) {
      cplx<ACC> a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        a[i] = As[kx * LD + ty + 16 * i];
        b[i] = Bs[kx * LD + tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {  // acc += conj(a) b, four fused multiply-adds
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(-a[i].y, b[j].x, acc[i][j].y);
        }
    }
    if (kCarry) {
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          two_sum_acc(chi[i][j].x, clo[i][j].x, (float)acc[i][j].x);
          two_sum_acc(chi[i][j].y, clo[i][j].y, (float)acc[i][j].y);
          acc[i][j] = mk<ACC>(0, 0);
        }
    }
    }
    __syncthreads();
  }
  double2* pz = part + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int m = tm + ty + 16 * i, n = tn + tx + 16 * j;
      if (m < M && n < N)
        pz[(size_t)m * N + n] =
            kCarry ? make_double2((double)chi[i][j].x + (double)clo[i][j].x, (double)chi[i][j].y + (double)clo[i][j].y)
                   : make_double2((double)acc[i][j].x, (double)acc[i][j].y);
    }
}

__global__ void k_reduce_parts(int M, int N, int nz, const double2* __restrict__ part, double2* __restrict__ C,
                               int ldc, int herm, int tile) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int m = idx / N, n = idx - m * N;
  const bool mirror = herm && (m / tile) > (n / tile);
  const size_t off = mirror ? (size_t)n * N + m : (size_t)m * N + n;
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < nz; ++z) s = cadd(s, part[(size_t)z * M * N + off]);
  C[(size_t)m * ldc + n] = mirror ? cconj(s) : s;
}

// micro-tile R (tile 16 R) for an M x N product: the least padded work, weighted by the micro-tile's cost
// per useful product (a thread's 2 R shared-memory loads feed 4 R^2 multiply-adds, so R = 2 spends about
// half its issue slots on loads)
static int pick_r(int M, int N, bool herm) {
  int best = 4;
  double best_work = 1e300;
  const double cost[5] = {0, 0, 1.5, 1.15, 1.0};
  for (int r = 4; r >= 2; --r) {
    const int t = 16 * r, tm = (M + t - 1) / t, tn = (N + t - 1) / t;
    const double tiles = herm ? tm * (tm + 1) / 2.0 : (double)tm * tn;
    const double work = tiles * t * t * cost[r];
    if (work < best_work * 0.999) {
      best_work = work;
      best = r;
    }
  }
  return best;
}

// K slices: the count nz (at most one per 256 of K, at most max_slices) that minimises the modelled
// makespan, ceil(tiles nz / 152) waves of CTAs sharing an SM times the steps (of `step` K values, the
// kernel's stage) of one slice; ties go to fewer slices (less partial-sum traffic).
static void split_k(int tiles, int K, size_t max_slices, int* nz_out, int* kslice_out, int resident = 1,
                    int step = 16) {
  const int steps = (K + step - 1) / step;
  int maxz = (K + 255) / 256;
  if ((size_t)maxz > max_slices) maxz = (int)max_slices;
  if (maxz < 1) maxz = 1;
  const long long slots = 152LL * (resident < 1 ? 1 : resident);  // CTAs resident at once
  long long best = -1;
  int best_nz = 1, best_steps = steps;
  for (int nz = 1; nz <= maxz; ++nz) {
    const int s = (steps + nz - 1) / nz;
    const int z = (steps + s - 1) / s;
    const long long waves = ((long long)tiles * z + slots - 1) / slots;
    const long long cost = waves * s;
    if (best < 0 || cost < best) {
      best = cost;
      best_nz = z;
      best_steps = s;
    }
  }
  *nz_out = best_nz;
  *kslice_out = best_steps * step;
}

// dynamic shared memory above the 48 KB default (the FP64 forms with R >= 3), set once per device
template <typename TA, typename TB, typename ACC, int R, bool CARRY>
static void cn_smem_attr(size_t sm) {
  static int dev_done = -1;
  int dev = 0;
  if (sm <= 48 * 1024 || cudaGetDevice(&dev) != cudaSuccess || dev == dev_done) return;
  if (cudaFuncSetAttribute(k_gemm_cn<TA, TB, ACC, R, CARRY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
      cudaSuccess)
    dev_done = dev;
}

template <typename TA, typename TB, typename ACC, bool CARRY>
static void launch_cn_r(int r, dim3 grid, cudaStream_t st, int M, int N, int K, int kslice, const cplx<TA>* A,
                        int lda, const cplx<TB>* B, int ldb, double2* part, int herm) {
  const size_t sm = (size_t)2 * 2 * CnStepK<ACC>::value * (16 * r + 1) * sizeof(cplx<ACC>);  // two stages of A, B
  if (r == 2) {
    cn_smem_attr<TA, TB, ACC, 2, CARRY>(sm);
    k_gemm_cn<TA, TB, ACC, 2, CARRY><<<grid, 256, sm, st>>>(M, N, K, kslice, A, lda, B, ldb, part, herm);
  } else if (r == 3) {
    cn_smem_attr<TA, TB, ACC, 3, CARRY>(sm);
    k_gemm_cn<TA, TB, ACC, 3, CARRY><<<grid, 256, sm, st>>>(M, N, K, kslice, A, lda, B, ldb, part, herm);
  } else {
    cn_smem_attr<TA, TB, ACC, 4, CARRY>(sm);
    k_gemm_cn<TA, TB, ACC, 4, CARRY><<<grid, 256, sm, st>>>(M, N, K, kslice, A, lda, B, ldb, part, herm);
  }
}

// resident CTAs per SM of the k_gemm_cn form (r, carry), from the occupancy calculator, cached per form
template <typename TA, typename TB, typename ACC, bool CARRY>
static int cn_resident_r(int r) {
  static int cached[5] = {0, 0, 0, 0, 0};
  if (r < 2 || r > 4) return 1;
  if (cached[r]) return cached[r];
  const size_t sm = (size_t)2 * 2 * CnStepK<ACC>::value * (16 * r + 1) * sizeof(cplx<ACC>);
  int nb = 1;
  cudaError_t e;
  if (r == 2) {
    cn_smem_attr<TA, TB, ACC, 2, CARRY>(sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_cn<TA, TB, ACC, 2, CARRY>, 256, sm);
  } else if (r == 3) {
    cn_smem_attr<TA, TB, ACC, 3, CARRY>(sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_cn<TA, TB, ACC, 3, CARRY>, 256, sm);
  } else {
    cn_smem_attr<TA, TB, ACC, 4, CARRY>(sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_cn<TA, TB, ACC, 4, CARRY>, 256, sm);
  }
  if (e != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cached[r] = nb;
  return nb;
}

template <typename TA, typename TB, typename ACC>
static int cn_resident(int r, bool carry) {
  return carry && sizeof(ACC) == 4 ? cn_resident_r<TA, TB, ACC, true>(r) : cn_resident_r<TA, TB, ACC, false>(r);
}

template <typename TA, typename TB, typename ACC>
static void launch_cn(int r, bool carry, dim3 grid, cudaStream_t st, int M, int N, int K, int kslice,
                      const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb, double2* part, int herm) {
  if (carry && sizeof(ACC) == 4)
    launch_cn_r<TA, TB, ACC, true>(r, grid, st, M, N, K, kslice, A, lda, B, ldb, part, herm);
  else
    launch_cn_r<TA, TB, ACC, false>(r, grid, st, M, N, K, kslice, A, lda, B, ldb, part, herm);
}

bool tc_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("PARO_NO_TC");
    return !(e && e[0] && e[0] != '0');
  }();
  return on;
}

int* tc_err_flag(Ctx* c) {
  if (!c->d_tc_err) {
    if (cudaMalloc(&c->d_tc_err, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream) != cudaSuccess) return nullptr;
  }
  return c->d_tc_err;
}

int tc_flag_readback(Ctx* c, const int** h) {
  *h = nullptr;
  if (!c->d_tc_err) return PARO_OK;
  void* p = nullptr;
  const int st = d2h_async(c, "tc_err", c->d_tc_err, sizeof(int), &p);
  *h = static_cast<const int*>(p);
  return st;
}

template <typename TA, typename TB, typename ACC>
int gemm_cn(Ctx* c, int M, int N, int K, const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb, double2* C,
            int ldc, bool herm, bool carry) {
  if (M <= 0 || N <= 0) return PARO_OK;
  if constexpr (sizeof(TA) == 4 && sizeof(TB) == 4 && sizeof(ACC) == 4) {
    if (!herm && !carry && K > 0 && c->tc_scope && tc_enabled()) {
      int* err = tc_err_flag(c);
      if (!err) return PARO_ERR_CUDA;
      cudaEvent_t ev = prof_begin(c);
      int st = gemm_cn_tc(c, M, N, K, A, lda, B, ldb, C, ldc, err);
      if (st) return st;
      prof_end(c, "k_gemm_cn_tc", ev);
      return PARO_OK;
    }
  }
  const int r = pick_r(M, N, herm), tile = 16 * r;
  const int tiles_m = (M + tile - 1) / tile, tiles_n = (N + tile - 1) / tile;
  const int tiles = herm ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
  int nz = 1, kslice = 16;
  split_k(tiles, K, (size_t)1 << 20, &nz, &kslice, cn_resident<TA, TB, ACC>(r, carry), CnStepK<ACC>::value);
  double2* part = static_cast<double2*>(ws_get(c, "gemm_parts", (size_t)nz * M * N * sizeof(double2)));
  if (!part) return PARO_ERR_CUDA;
  if (K == 0) {
    PARO_CU(c, cudaMemsetAsync(part, 0, (size_t)M * N * sizeof(double2), c->stream));
  } else {
    cudaEvent_t ev = prof_begin(c);
    launch_cn<TA, TB, ACC>(r, carry, dim3(tiles_n, tiles_m, nz), c->stream, M, N, K, kslice, A, lda, B, ldb,
                           part, herm ? 1 : 0);
    PARO_LAUNCH(c, "k_gemm_cn");
    prof_end(c, sizeof(ACC) == 8 ? "k_gemm_cn<f64>" : "k_gemm_cn<f32>", ev);
  }
  k_reduce_parts<<<(M * N + 255) / 256, 256, 0, c->stream>>>(M, N, K == 0 ? 1 : nz, part, C, ldc, herm ? 1 : 0,
                                                             tile);
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
  const int r = pick_r(M, N, false), tile = 16 * r;
  const int tiles_m = (M + tile - 1) / tile, tiles_n = (N + tile - 1) / tile;
  int nz = 1, kslice = 16;
  split_k(tiles_m * tiles_n, K, part_elems / slice, &nz, &kslice, 1, CnStepK<ACC>::value);
  launch_cn<TA, TB, ACC>(r, false, dim3(tiles_n, tiles_m, nz), c->stream, M, N, K, kslice, A, lda, B, ldb, part,
                         0);
  PARO_LAUNCH(c, "k_gemm_cn");
  k_reduce_parts<<<(M * N + 255) / 256, 256, 0, c->stream>>>(M, N, nz, part, C, ldc, 0, tile);
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

// FP32 form: Y = beta Y + W^T X with every output row of a (16 RM)-row block in one CTA, so the long X
// (K x N_pw) is read once per row block. 256 threads = 16 x 16, thread (ty, tx) holds rows ty + 16 i
// (i < RM) and columns tx + 16 j (j < RN): RM + RN shared-memory loads per RM RN complex products.
// Wf[k][m] = (float)(s_k W(k, m)), K x M: the small matrix converted once per call, because a conversion
// or product in FP64 per staged element would occupy GB300's FP64 pipe longer than the product's FMAs
__global__ void k_w_to_f32(int M, int K, const double2* __restrict__ W, int ldw, int wt,
                           const double* __restrict__ s, float2* __restrict__ Wf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M * K; i += gridDim.x * blockDim.x) {
    const int k = i / M, m = i - k * M;
    double2 w = wt ? W[(size_t)m * ldw + k] : W[(size_t)k * ldw + m];
    if (s) w = cscale(w, s[k]);
    Wf[i] = make_float2((float)w.x, (float)w.y);
  }
}

// Thread (ty, tx) holds rows tm + RM ty + i (i < RM) and columns tn + tx + 16 j (j < RN), so a warp
// (two ty) holds 2 RM consecutive rows. LW: W(k, m) = 0 for k > m; a warp skips the K steps that lie
// beyond its last row, and the CTA those beyond its tile's last row.
template <int RM, int RN, bool LW = false>
__global__ void __launch_bounds__(256) k_gemm_wx32(int M, int N, int K, const float2* __restrict__ Wf,
                                                   const float2* __restrict__ X, int ldx, float2* __restrict__ Y,
                                                   int ldy, float beta) {
  constexpr int TM = 16 * RM, TN = 16 * RN, STG = 16 * (TM + TN);  // float2 per stage buffer
  extern __shared__ __align__(16) float2 wx_smem[];                // three stages: Ws[16][TM], Xs[16][TN]
  const int tm = blockIdx.y * TM, tn = blockIdx.x * TN;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  // the K step k0 into stage buffer st by asynchronous 8-byte copies (zero-filled outside the matrices)
  auto stage = [&](int k0, int st) {
    float2* Ws = wx_smem + st * STG;
    float2* Xs = Ws + 16 * TM;
    for (int i = tid; i < 16 * TM; i += 256) {
      const int kx = i / TM, r = i - kx * TM, gk = k0 + kx, gm = tm + r;
      const bool in = gk < K && gm < M;
      cp_async8(Ws + i, in ? Wf + (size_t)gk * M + gm : Wf, in ? 8 : 0);
    }
    for (int i = tid; i < 16 * TN; i += 256) {
      const int kx = i / TN, cc = i - kx * TN, gk = k0 + kx, gn = tn + cc;
      const bool in = gk < K && gn < N;
      cp_async8(Xs + i, in ? X + (size_t)gk * ldx + gn : X, in ? 8 : 0);
    }
    cp_async_commit();
  };
  float2 acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const int nk = LW ? min((K + 15) / 16, (tm + TM + 15) / 16) : (K + 15) / 16;
  // a ring of three stages, one barrier per stage: the barrier that publishes stage kt also marks stage
  // kt - 1 as read, and its buffer takes stage kt + 2
  if (nk > 0) stage(0, 0);
  if (nk > 1) stage(16, 1);
  const int warp_last_row = tm + RM * (ty | 1) + RM - 1;
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) cp_async_wait<1>();  // stages committed so far: kt + 2 (kt + 1 at the last)
    else cp_async_wait<0>();
    __syncthreads();
    if (kt + 2 < nk) stage(16 * (kt + 2), (kt + 2) % 3);
    const float2* Ws = wx_smem + (kt % 3) * STG;
    const float2* Xs = Ws + 16 * TM;
    if (!LW || 16 * kt <= warp_last_row)
#pragma unroll 4
    for (int kx = 0; kx < 16; ++kx) {
      float2 x[RN], w[RM];
#pragma unroll
      for (int j = 0; j < RN; ++j) x[j] = Xs[kx * TN + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i) w[i] = Ws[kx * TM + RM * ty + i];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          acc[i][j].x = fmaf(w[i].x, x[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-w[i].y, x[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(w[i].x, x[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(w[i].y, x[j].x, acc[i][j].y);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int m = tm + RM * ty + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int n = tn + tx + 16 * j;
      if (n >= N) continue;
      float2 v = acc[i][j];
      if (beta != 0.f) {
        const float2 o = Y[(size_t)m * ldy + n];
        v = make_float2(fmaf(beta, o.x, v.x), fmaf(beta, o.y, v.y));
      }
      Y[(size_t)m * ldy + n] = v;
    }
  }
}

// launch of k_gemm_wx32: RM = 9 (144-row blocks) unless M fits 64 rows; RN (32 or 64 columns) with the
// smaller makespan in waves of 152 SMs x resident CTAs
static int launch_wx32(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s,
                       const float2* X, int ldx, float2* Y, int ldy, double beta, float2* Wf, bool lower) {
  const bool big = M > 64;
  const int tm = big ? 144 : 64;
  const int mt = (M + tm - 1) / tm;
  const long long s2 = (long long)mt * ((N + 31) / 32), s4 = (long long)mt * ((N + 63) / 64);
  // resident CTAs per SM by register use: about 3 (RN = 2) and 2 (RN = 4) at RM = 9
  const long long w2 = (s2 + 3 * 152 - 1) / (3 * 152) * 2, w4 = (s4 + 2 * 152 - 1) / (2 * 152) * 4;
  const bool rn4 = w4 < w2;
  const dim3 grid((N + (rn4 ? 63 : 31)) / (rn4 ? 64 : 32), mt);
  const float fb = (float)beta;
  if (!Wf) Wf = static_cast<float2*>(ws_get(c, "wx32_w", (size_t)M * K * sizeof(float2)));
  if (!Wf) return PARO_ERR_CUDA;
  if (K > 0) {
    k_w_to_f32<<<std::min((M * K + 255) / 256, 304), 256, 0, c->stream>>>(M, K, W, ldw, wt ? 1 : 0, s, Wf);
    PARO_LAUNCH(c, "k_w_to_f32");
  }
  const int rm = big ? 9 : 4, rn = rn4 ? 4 : 2;
  const size_t sm = (size_t)3 * 16 * 16 * (rm + rn) * sizeof(float2);  // three stages
  static int attr_dev = -1;  // dynamic shared memory above 48 KB, set per device
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (attr_dev != dev) {
    for (const void* f : {(const void*)k_gemm_wx32<9, 4>, (const void*)k_gemm_wx32<9, 4, true>,
                          (const void*)k_gemm_wx32<9, 2>, (const void*)k_gemm_wx32<9, 2, true>,
                          (const void*)k_gemm_wx32<4, 4>, (const void*)k_gemm_wx32<4, 2>})
      PARO_CU(c, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr_dev = dev;
  }
  if (big && lower) {
    if (rn4) k_gemm_wx32<9, 4, true><<<grid, 256, sm, c->stream>>>(M, N, K, Wf, X, ldx, Y, ldy, fb);
    else k_gemm_wx32<9, 2, true><<<grid, 256, sm, c->stream>>>(M, N, K, Wf, X, ldx, Y, ldy, fb);
  } else if (big) {
    if (rn4) k_gemm_wx32<9, 4><<<grid, 256, sm, c->stream>>>(M, N, K, Wf, X, ldx, Y, ldy, fb);
    else k_gemm_wx32<9, 2><<<grid, 256, sm, c->stream>>>(M, N, K, Wf, X, ldx, Y, ldy, fb);
  } else {
    if (rn4) k_gemm_wx32<4, 4><<<grid, 256, sm, c->stream>>>(M, N, K, Wf, X, ldx, Y, ldy, fb);
    else k_gemm_wx32<4, 2><<<grid, 256, sm, c->stream>>>(M, N, K, Wf, X, ldx, Y, ldy, fb);
  }
  PARO_LAUNCH(c, "k_gemm_wx32");
  return PARO_OK;
}

template <typename TX, typename TY>
int gemm_wx(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s, const cplx<TX>* X,
            int ldx, cplx<TY>* Y, int ldy, double beta, float2* wf, bool lower) {
  if (M <= 0 || N <= 0) return PARO_OK;
  if constexpr (sizeof(TX) == 4 && sizeof(TY) == 4) {
    if (c->tc_scope && tc_enabled()) {
      int* err = tc_err_flag(c);
      if (!err) return PARO_ERR_CUDA;
      cudaEvent_t ev = prof_begin(c);
      int st = gemm_wx_tc(c, M, N, K, W, ldw, wt, s, X, ldx, Y, ldy, beta, err);
      if (st) return st;
      prof_end(c, "k_gemm_wx_tc", ev);
      return PARO_OK;
    }
    cudaEvent_t ev = prof_begin(c);
    int st = launch_wx32(c, M, N, K, W, ldw, wt, s, X, ldx, Y, ldy, beta, wf, lower);
    if (st) return st;
    prof_end(c, "k_gemm_wx<f32>", ev);
    return PARO_OK;
  }
  cudaEvent_t ev = prof_begin(c);
  k_gemm_wx<TX, TY><<<dim3((N + 63) / 64, (M + 31) / 32), 256, 0, c->stream>>>(M, N, K, W, ldw, wt ? 1 : 0, s, X,
                                                                               ldx, Y, ldy, beta);
  PARO_LAUNCH(c, "k_gemm_wx");
  prof_end(c, sizeof(TY) == 8 ? "k_gemm_wx<f64>" : "k_gemm_wx<f32>", ev);
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Cholesky S = L L^H and G = conj(L)^{-1} (cooperative, many CTAs). Right-looking: at step j every CTA
// reads the pivot S_jj of the updated matrix W, stores column j of L and applies the rank-1 update
// W_ik -= W_ij conj(W_kj) / W_jj to its share of the trailing lower triangle; a grid barrier closes
// each step. Then G's columns are independent forward substitutions conj(L) g_j = e_j, one warp per
// column. info[0] = 0, or 1 + the first column whose pivot is not positive.
__global__ void __launch_bounds__(256) k_chol(int n, const double2* __restrict__ S, double2* __restrict__ W,
                                              double2* __restrict__ Lm, double2* __restrict__ G, unsigned* bar,
                                              int* err, int* info) {
  const int gth = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int gwarp = gth >> 5, nwarp = nth >> 5;
  for (size_t idx = gth; idx < (size_t)n * n; idx += nth) {
    __stcg(&W[idx], S[idx]);
    __stcg(&Lm[idx], make_double2(0.0, 0.0));
  }
  if (!grid_barrier(bar, err)) return;
  for (int j = 0; j < n; ++j) {
    double djj = __ldcg(&W[(size_t)j * n + j]).x;
    if (!(djj > 0.0) || !isfinite(djj)) {
      if (gth == 0) atomicCAS(info, 0, j + 1);
      djj = 1.0;
    }
    const double ljj = sqrt(djj);
    const int m = n - j - 1;
    for (int i = gth; i < m; i += nth)
      __stcg(&Lm[(size_t)(j + 1 + i) * n + j], cscale(__ldcg(&W[(size_t)(j + 1 + i) * n + j]), 1.0 / ljj));
    if (gth == 0) __stcg(&Lm[(size_t)j * n + j], make_double2(ljj, 0.0));
    // trailing lower triangle (i >= k > j), element count m (m + 1) / 2
    const size_t tot = (size_t)m * (m + 1) / 2;
    const double inv = 1.0 / djj;
    for (size_t t = gth; t < tot; t += nth) {
      // t -> (i, k) with 0 <= k <= i < m, row-major over the lower triangle
      int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
      while ((size_t)i * (i + 1) / 2 > t) --i;
      while ((size_t)(i + 1) * (i + 2) / 2 <= t) ++i;
      const int k = (int)(t - (size_t)i * (i + 1) / 2);
      const double2 wi = __ldcg(&W[(size_t)(j + 1 + i) * n + j]);
      const double2 wk = __ldcg(&W[(size_t)(j + 1 + k) * n + j]);
      double2* p = &W[(size_t)(j + 1 + i) * n + (j + 1 + k)];
      double2 v = __ldcg(p);
      v.x -= (wi.x * wk.x + wi.y * wk.y) * inv;
      v.y -= (wi.y * wk.x - wi.x * wk.y) * inv;
      __stcg(p, v);
    }
    if (!grid_barrier(bar, err)) return;
  }
  // G = conj(L)^{-1}: column j solves conj(L) g = e_j; lanes share the inner sums
  for (int j = gwarp; j < n; j += nwarp) {
    for (int i = lane; i < j; i += 32) G[(size_t)i * n + j] = make_double2(0.0, 0.0);
    if (lane == 0) G[(size_t)j * n + j] = make_double2(1.0 / __ldcg(&Lm[(size_t)j * n + j]).x, 0.0);
    __syncwarp();
    for (int i = j + 1; i < n; ++i) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = j + lane; k < i; k += 32) s = cadd(s, cmul(cconj(__ldcg(&Lm[(size_t)i * n + k])), G[(size_t)k * n + j]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) G[(size_t)i * n + j] = cscale(s, -1.0 / __ldcg(&Lm[(size_t)i * n + i]).x);
      __syncwarp();
    }
  }
}

int coop_grid(Ctx* c, const void* kernel, int threads, size_t smem, int cap, int* grid);  // k_eigh.cu

// Cholesky S = L L^H and G = conj(L)^{-1} on one thread-block cluster of C CTAs, row g of [S | I] in
// CTA g mod C. Gaussian elimination without pivoting (stable for Hermitian positive definite S): step j
// subtracts m_ij = a_ij / a_jj times pivot row j from every row i > j, in both halves. That leaves the
// diagonal D of S = L_u D L_u^H on the left and L_u^{-1} on the right (L_u unit lower triangular), so
// L^{-1} = D^{-1/2} L_u^{-1}. The trailing left block stays Hermitian, so only its lower triangle is kept
// (a third less FP64 work than the full rows): the pivot row's left part a_jk (k > j) is read as
// conj(a_kj), column j of the rows below. After step j - 1 each CTA pushes column j of its rows, and
// the owner of row j the right half of row j, into every CTA's shared memory (double-buffered by the
// parity of j), so each step reads its pivot locally; one cluster barrier per column orders the steps.
// info: first column + 1 with a_jj <= 0 (the elimination then continues with a_jj = 1).
__global__ void __launch_bounds__(1024) k_chol_cluster(int n, const double2* __restrict__ s, double2* __restrict__ g,
                                                       int* __restrict__ info, const int* __restrict__ skip) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  if (skip != nullptr && *skip) {  // the factor is already formed (k_orth_first_order); every CTA leaves at once
    if (q == 0 && threadIdx.x == 0) *info = 0;
    return;
  }
  const int R = (n + C - 1) / C, W2 = 2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* rows = reinterpret_cast<double2*>(smem_raw);  // R x 2n: [a_i | b_i]
  double2* pivb = rows + (size_t)R * W2;                 // 2 x 2n: pivot row of step j in pivb[j & 1]
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (tid == 0) s_bad = 0;
  for (size_t idx = tid; idx < (size_t)R * W2; idx += blockDim.x) {
    const int r = (int)(idx / W2), k = (int)(idx - (size_t)r * W2), gi = q + C * r;
    double2 v = make_double2(0.0, 0.0);
    if (gi < n) v = k < n ? s[(size_t)gi * n + k] : make_double2(k - n == gi ? 1.0 : 0.0, 0.0);
    rows[idx] = v;
  }
  // pivot data of step c into every CTA: conj(a_kc) of this CTA's rows k >= c (left part, at index k),
  // and, from the owner of row c, its right half b_ck (k <= c, at index n + k)
  auto push = [&](int c) {
    double2* dst = pivb + (c & 1) * W2;
    const int rc0 = (c > q) ? (c - q + C - 1) / C : 0;  // first local row with g >= c
    const int nl = R - rc0;
    for (int t = tid; t < nl * C; t += blockDim.x) {
      const int r = rc0 + t / C, tgt = t - (t / C) * C, gi = q + C * r;
      if (gi >= n) continue;
      double2* rd = cl.map_shared_rank(dst, tgt);
      rd[gi] = cconj(rows[(size_t)r * W2 + c]);
    }
    if (c % C == q) {
      const double2* rowc = rows + (size_t)(c / C) * W2 + n;
      for (int t = tid; t < (c + 1) * C; t += blockDim.x) {
        const int k = t / C, tgt = t - k * C;
        double2* rd = cl.map_shared_rank(dst, tgt);
        rd[n + k] = rowc[k];
      }
    }
  };
  cl.sync();  // every CTA of the cluster is running (and has its rows) before shared memory is written remotely
  push(0);
  cl.sync();
  for (int j = 0; j < n; ++j) {
    const double2* piv = pivb + (j & 1) * W2;
    double ajj = piv[j].x;
    if (!(ajj > 0.0) || !isfinite(ajj)) {
      if (tid == 0 && s_bad == 0) s_bad = j + 1;
      ajj = 1.0;
    }
    const double inv = 1.0 / ajj;
    const int r0 = (j + 1 > q) ? (j + 1 - q + C - 1) / C : 0;  // first local row with g > j
    for (int r = r0 + warp; r < R; r += nwarp) {
      const int gi = q + C * r;
      if (gi >= n) break;
      double2* row = rows + (size_t)r * W2;
      const double2 m = cscale(row[j], inv);
      for (int k = j + 1 + lane; k <= gi; k += 32) row[k] = csub(row[k], cmul(m, piv[k]));
      for (int k = lane; k <= j; k += 32) row[n + k] = csub(row[n + k], cmul(m, piv[n + k]));
    }
    if (j + 1 < n) {
      __syncthreads();  // this CTA's rows are updated for step j
      push(j + 1);
    }
    cl.sync();
  }
  for (size_t idx = tid; idx < (size_t)R * n; idx += blockDim.x) {
    const int r = (int)(idx / n), k = (int)(idx - (size_t)r * n), gi = q + C * r;
    if (gi >= n) continue;
    const double d = rows[(size_t)r * W2 + gi].x;
    const double2 b = rows[(size_t)r * W2 + n + k];
    g[(size_t)gi * n + k] = (k <= gi && d > 0.0) ? cscale(cconj(b), 1.0 / sqrt(d)) : make_double2(0.0, 0.0);
  }
  if (q == 0 && tid == 0) *info = s_bad;
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

// Blocked form of the same factorisation (right-looking block Cholesky, blocks of C columns, row g in
// CTA g mod C, so each CTA owns exactly one row of every block). Block J (columns c0 .. c1 - 1) takes
// two cluster barriers instead of one per column:
//   every CTA factors the pushed diagonal block D = A_JJ itself by elimination of [D | I] (giving
//   D = L_u diag(d) L_u^H and L_u^{-1}, so L_JJ^{-1} = diag(d)^{-1/2} L_u^{-1});
//   each CTA forms the panel rows L_iJ = A_iJ L_JJ^{-H} of its rows below the block, and the owner
//   of diagonal row t the finished row t of L^{-1}, (L_JJ^{-1} B_J)_t, where B_J holds the rows of
//   the block after the earlier block updates of the right half; both go to every CTA; barrier;
//   each CTA updates its rows below: a_ik -= L_iJ conj(L_kJ) (lower triangle), b_ik -= L_iJ (L^{-1})_Jk;
//   the owners of the next block push its diagonal rows; barrier.
// Shared memory (double2): rows R x 2n ([a_i | b_i]), panel C x n (pan[s][k] = L_k,c0+s), linv C x n
// (rows of L^{-1} of the block), brow C x n (pushed B_J), dblk, dinv C x C. info as k_chol_cluster.
// acc + a b and acc + a conj(b) as four FMAs
__device__ __forceinline__ double2 zfma(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 zfma_conj(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
  return acc;
}

__global__ void __launch_bounds__(512) k_chol_blocked(int n, const double2* __restrict__ s, double2* __restrict__ g,
                                                      int* __restrict__ info, const int* __restrict__ skip) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  if (skip != nullptr && *skip) {  // the factor is already formed (k_orth_first_order); every CTA leaves at once
    if (q == 0 && threadIdx.x == 0) *info = 0;
    return;
  }
  const int R = (n + C - 1) / C, W2 = 2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* rows = reinterpret_cast<double2*>(smem_raw);  // R x 2n
  double2* pan = rows + (size_t)R * W2;                  // C x n
  double2* linv = pan + (size_t)C * n;                   // C x n
  double2* brow = linv + (size_t)C * n;                  // C x n
  double2* dblk = brow + (size_t)C * n;                  // C x C (lower)
  double2* dinv = dblk + C * C;                          // C x C (lower)
  __shared__ double s_rcp[32], s_isq[32];
  __shared__ int s_bad, s_off[64];
  __shared__ unsigned char s_trow[16 * 17 / 2], s_tcol[16 * 17 / 2];  // lower triangle of order <= 16
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) s_bad = 0;
  if (tid < 16) {
    const int t = tid;
    for (int l = 0; l <= t; ++l) {
      s_trow[t * (t + 1) / 2 + l] = (unsigned char)t;
      s_tcol[t * (t + 1) / 2 + l] = (unsigned char)l;
    }
  }
  for (size_t idx = tid; idx < (size_t)R * W2; idx += nth) {
    const int r = (int)(idx / W2), k = (int)(idx - (size_t)r * W2), gi = q + C * r;
    double2 v = make_double2(0.0, 0.0);
    if (gi < n) v = k < n ? s[(size_t)gi * n + k] : make_double2(k - n == gi ? 1.0 : 0.0, 0.0);
    rows[idx] = v;
  }
  // this CTA's row of the block starting at c: diagonal-block part and B part into every CTA
  auto push_diag = [&](int c) {
    const int gi = c + q;
    if (gi >= n) return;
    const int t = q, c1 = min(c + C, n);
    const double2* row = rows + (size_t)(gi / C) * W2;
    for (int u = tid; u < (t + 1 + c1) * C; u += nth) {
      const int e = u / C, tgt = u - e * C;
      if (e <= t) cl.map_shared_rank(dblk, tgt)[t * C + e] = row[c + e];
      else cl.map_shared_rank(brow, tgt)[(size_t)t * n + (e - t - 1)] = row[n + e - t - 1];
    }
  };
  cl.sync();  // every CTA of the cluster is running before shared memory is written remotely
  __syncthreads();
  push_diag(0);
  cl.sync();
  for (int c0 = 0; c0 < n; c0 += C) {
    const int c1 = min(c0 + C, n), w = c1 - c0;
    // ---- diagonal block: elimination of [D | I], redundantly in every CTA ----
    for (int u = tid; u < w * w; u += nth) {
      const int t = u / w, e = u - t * w;
      dinv[t * C + e] = make_double2(t == e ? 1.0 : 0.0, 0.0);
    }
    if (tid == 0) {
      double d = dblk[0].x;
      if (!(d > 0.0) || !isfinite(d)) {
        if (s_bad == 0) s_bad = c0 + 1;
        d = 1.0;
        dblk[0] = make_double2(1.0, 0.0);
      }
      s_rcp[0] = 1.0 / d;
    }
    __syncthreads();
    // Step j updates rows t > j: t - j entries of the left block (columns j + 1 .. t) and j + 1 of the
    // right (columns 0 .. j), t + 1 in all. The entries of all rows are packed densely onto consecutive
    // threads (a warp's FP64 instruction costs the same with idle lanes): entry u of step j is entry
    // v = u + (j + 1)(j + 2) / 2 of the row-major lower triangle, row s_trow[v], position s_tcol[v].
    for (int j = 0; j + 1 < w; ++j) {
      const int v0 = (j + 1) * (j + 2) / 2, nitem = w * (w + 1) / 2 - v0;
      if (tid < nitem) {
        const int v = tid + v0, t = s_trow[v], l = s_tcol[v];
        const double2 a = dblk[t * C + j];
        const double r = s_rcp[j];
        const double2 m = make_double2(a.x * r, a.y * r);
        if (l < t - j) {  // x -= m conj(y)
          const int e = j + 1 + l;
          const double2 y = dblk[e * C + j];
          double2 x = dblk[t * C + e];
          x.x = fma(-m.x, y.x, x.x);
          x.x = fma(-m.y, y.y, x.x);
          x.y = fma(-m.y, y.x, x.y);
          x.y = fma(m.x, y.y, x.y);
          dblk[t * C + e] = x;
          if (e == t && t == j + 1) {  // the next pivot is final
            double d = x.x;
            if (!(d > 0.0) || !isfinite(d)) {
              if (s_bad == 0) s_bad = c0 + t + 1;
              d = 1.0;
              dblk[t * C + t] = make_double2(1.0, 0.0);
            }
            s_rcp[t] = 1.0 / d;
          }
        } else {  // x -= m y
          const int e = l - (t - j);
          const double2 y = dinv[j * C + e];
          double2 x = dinv[t * C + e];
          x.x = fma(-m.x, y.x, x.x);
          x.x = fma(m.y, y.y, x.x);
          x.y = fma(-m.x, y.y, x.y);
          x.y = fma(-m.y, y.x, x.y);
          dinv[t * C + e] = x;
        }
      }
      __syncthreads();
    }
    if (tid < w) s_isq[tid] = 1.0 / sqrt(dblk[tid * C + tid].x);
    __syncthreads();
    // ---- panel rows of this CTA below the block, and the finished row t = q of L^{-1} ----
    const int rb = (c1 > q) ? (c1 - q + C - 1) / C : 0;  // first local row with g >= c1
    const int nbelow = max(0, min(R, (n - q + C - 1) / C) - rb);
    const int n3a = nbelow * w;
    const int n3b = (q < w) ? c1 : 0;
    for (int u = tid; u < n3a + n3b; u += nth) {
      if (u < n3a) {  // s-major: the entries of a warp have inner sums of similar length
        const int sidx = u / nbelow, r = rb + (u - sidx * nbelow), gi = q + C * r;
        const double2* a = rows + (size_t)r * W2 + c0;
        double2 acc = make_double2(0.0, 0.0);
        for (int t = 0; t <= sidx; ++t) acc = zfma_conj(acc, a[t], dinv[sidx * C + t]);
        acc = cscale(acc, s_isq[sidx]);
        for (int tgt = 0; tgt < C; ++tgt) cl.map_shared_rank(pan, tgt)[(size_t)sidx * n + gi] = acc;
      } else {
        const int k = u - n3a, t = q;
        double2 acc = make_double2(0.0, 0.0);
        for (int e = 0; e <= t; ++e) acc = zfma(acc, dinv[t * C + e], brow[(size_t)e * n + k]);
        acc = cscale(acc, s_isq[t]);
        rows[(size_t)((c0 + t) / C) * W2 + n + k] = acc;  // final row c0 + t of L^{-1}
        for (int tgt = 0; tgt < C; ++tgt) cl.map_shared_rank(linv, tgt)[(size_t)t * n + k] = acc;
      }
    }
    cl.sync();
    if (c1 >= n) break;
    // ---- update of this CTA's rows below the block: k < c1 in the right half, c1 <= k <= g on the left ----
    if (tid == 0) {
      int o = 0;
      for (int r = 0; r < nbelow; ++r) {
        s_off[r] = o;
        o += q + C * (rb + r) + 1;
      }
      s_off[nbelow] = o;
    }
    __syncthreads();
    const int nitem = s_off[nbelow];
    for (int u = tid; u < nitem; u += nth) {
      int r = 0;
      while (s_off[r + 1] <= u) ++r;
      const int k = u - s_off[r], lr = rb + r, gi = q + C * lr;
      double2* row = rows + (size_t)lr * W2;
      double2 acc = make_double2(0.0, 0.0);
      if (k < c1) {
        for (int e = 0; e < w; ++e) acc = zfma(acc, pan[(size_t)e * n + gi], linv[(size_t)e * n + k]);
        row[n + k] = csub(row[n + k], acc);
      } else {
        for (int e = 0; e < w; ++e) acc = zfma_conj(acc, pan[(size_t)e * n + gi], pan[(size_t)e * n + k]);
        row[k] = csub(row[k], acc);
      }
    }
    __syncthreads();
    push_diag(c1);
    cl.sync();
  }
  for (size_t idx = tid; idx < (size_t)R * n; idx += nth) {
    const int r = (int)(idx / n), k = (int)(idx - (size_t)r * n), gi = q + C * r;
    if (gi >= n) continue;
    g[(size_t)gi * n + k] = k <= gi ? cconj(rows[(size_t)r * W2 + n + k]) : make_double2(0.0, 0.0);
  }
  if (q == 0 && tid == 0) *info = s_bad;
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

static size_t chol_blocked_smem(int n, int C) {
  const int R = (n + C - 1) / C;
  return ((size_t)R * 2 * n + 3 * (size_t)C * n + 2 * (size_t)C * C) * sizeof(double2);
}

// Launch shape of the cluster Cholesky for order n: the blocked kernel where its shared memory fits,
// else the column-by-column one; cluster size 16, else 8. kind 0: neither fits (cooperative fallback).
static int chol_cluster_shape(Ctx* c, int n, Ctx::CholShape* out) {
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (c->chol_shape.n == n && c->chol_shape.dev == dev) {
    *out = c->chol_shape;
    return PARO_OK;
  }
  const size_t cap = 220 * 1024;
  PARO_CU(c, cudaFuncSetAttribute(k_chol_blocked, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  PARO_CU(c, cudaFuncSetAttribute(k_chol_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  PARO_CU(c, cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  PARO_CU(c, cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  Ctx::CholShape sh;
  sh.n = n;
  sh.dev = dev;
  for (int kind : {1, 2}) {
    for (int C : {16, 8}) {
      const int R = (n + C - 1) / C;
      size_t sm;
      int thr;
      const void* kern;
      if (kind == 1) {  // blocked: s_off holds R + 1 row offsets
        sm = chol_blocked_smem(n, C);
        thr = 512;
        kern = (const void*)k_chol_blocked;
        if (sm > cap || R > 62) continue;
      } else {
        sm = ((size_t)R * 2 * n + 4 * (size_t)n) * sizeof(double2);  // rows, two pivot buffers
        thr = 32 * (R < 4 ? 4 : (R > 32 ? 32 : R));
        kern = (const void*)k_chol_cluster;
        if (sm > 200 * 1024) continue;
      }
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(thr);
      cfg.dynamicSmemBytes = sm;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (nclusters >= 1) {
        sh.kind = kind;
        sh.cls = C;
        sh.thr = thr;
        sh.smem = sm;
        c->chol_shape = *out = sh;
        return PARO_OK;
      }
    }
  }
  c->chol_shape = *out = sh;
  return PARO_OK;
}

int chol_check(Ctx* c) {
  int bad = 0;
  for (const std::string& nm : c->chol_pending) {
    int st = pinned_wait(c, nm.c_str());
    if (st) return st;
    const int h = *static_cast<const int*>(c->pinned[nm].h);
    if (h && !bad) bad = h;
  }
  c->chol_pending.clear();
  if (bad) return fail(c, PARO_ERR_BREAKDOWN, "Cholesky pivot <= 0 at column " + std::to_string(bad - 1));
  return PARO_OK;
}

// First-order inverse Cholesky factor of a Gram matrix close to the identity. With S = I + E = L L^H and
// F = strictly lower(E) + diag(E) / 2, L = I + F + O(E^2), so G = conj(L)^{-1} = I - conj(F) + O(E^2), and the
// rows G X are orthonormal up to about 3 ||E||^2. Every CTA forms ||E||_F (in FP32: it only decides the
// path, and one CTA's FP64 pipe would take tens of microseconds over the n^2 entries) in the same order,
// so all of them reach the same verdict; when it is at most tol each writes its rows of G (lower
// triangular, as the Cholesky kernels do) and CTA 0 sets *use, else *use = 0 and G is left alone.
__global__ void __launch_bounds__(1024) k_orth_first_order(int n, const double2* __restrict__ s,
                                                           double2* __restrict__ g, double tol, int* __restrict__ use,
                                                           double* __restrict__ enorm) {
  __shared__ float red[32];
  __shared__ int s_use;
  float acc = 0.f;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i / n, k = i - r * n;
    const double2 v = s[i];
    const float x = r == k ? (float)(v.x - 1.0) : (float)v.x, y = (float)v.y;
    acc = fmaf(x, x, fmaf(y, y, acc));
  }
  acc = block_sumf(acc, red);
  if (threadIdx.x == 0) {
    const float e = sqrtf(acc);
    s_use = (double)e <= tol ? 1 : 0;
    if (blockIdx.x == 0) {
      *enorm = (double)e;
      *use = s_use;
    }
  }
  __syncthreads();
  if (!s_use) return;
  const int r0 = (int)((long long)n * blockIdx.x / gridDim.x), r1 = (int)((long long)n * (blockIdx.x + 1) / gridDim.x);
  for (int i = r0 * n + threadIdx.x; i < r1 * n; i += blockDim.x) {
    const int r = i / n, k = i - r * n;
    const double2 v = s[i];
    // -conj(v) below the diagonal: a sign flip of the real part's bits, no FP64 arithmetic
    g[i] = k > r ? make_double2(0.0, 0.0)
                 : k == r ? make_double2(1.5 - 0.5 * v.x, 0.0)
                          : make_double2(__longlong_as_double(__double_as_longlong(v.x) ^ (long long)0x8000000000000000ULL),
                                         v.y);
  }
}

int chol_cluster_available(Ctx* c, int n, bool* avail) {
  Ctx::CholShape sh;
  const int st = chol_cluster_shape(c, n, &sh);
  *avail = st == PARO_OK && sh.kind > 0;
  return st;
}

int orth_first_order(Ctx* c, int n, const double2* s, double2* g, double tol, int** use_dev) {
  int* use = static_cast<int*>(ws_get(c, "orth_first_use", sizeof(int)));
  double* enorm = static_cast<double*>(ws_get(c, "orth_first_enorm", sizeof(double)));
  if (!use || !enorm) return PARO_ERR_CUDA;
  k_orth_first_order<<<16, 1024, 0, c->stream>>>(n, s, g, tol, use, enorm);
  PARO_LAUNCH(c, "k_orth_first_order");
  *use_dev = use;
  return PARO_OK;
}

int chol_inv(Ctx* c, int n, const double2* s, double2* g, bool defer, const int* skip) {
  {
    Ctx::CholShape sh;
    int st;
    if ((st = chol_cluster_shape(c, n, &sh))) return st;
    if (sh.kind > 0) {
      int* flags = static_cast<int*>(ws_get(c, "chol_flags", 8 * sizeof(int)));
      if (!flags) return PARO_ERR_CUDA;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = sh.cls;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(sh.cls);
      cfg.blockDim = dim3(sh.thr);
      cfg.dynamicSmemBytes = sh.smem;
      cfg.stream = c->stream;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaEvent_t ev = prof_begin(c);
      if (sh.kind == 1) PARO_CU(c, cudaLaunchKernelEx(&cfg, k_chol_blocked, n, s, g, flags, skip));
      else PARO_CU(c, cudaLaunchKernelEx(&cfg, k_chol_cluster, n, s, g, flags, skip));
      ++c->launches;
      prof_end(c, "k_chol_cluster", ev);
      if (defer) {  // the flag comes back without waiting; chol_check() reads it
        const std::string nm = "chol_flag_" + std::to_string(c->chol_pending.size());
        if ((st = d2h_async(c, nm.c_str(), flags, sizeof(int), nullptr))) return st;
        c->chol_pending.push_back(nm);
        return PARO_OK;
      }
      int h = 0;
      PARO_CU(c, cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      PARO_CU(c, cudaStreamSynchronize(c->stream));
      if (h) return fail(c, PARO_ERR_BREAKDOWN, "Cholesky pivot <= 0 at column " + std::to_string(h - 1));
      return PARO_OK;
    }
  }
  double2* W = static_cast<double2*>(ws_get(c, "chol_W", (size_t)n * n * sizeof(double2)));
  double2* L = static_cast<double2*>(ws_get(c, "chol_L", (size_t)n * n * sizeof(double2)));
  int* flags = static_cast<int*>(ws_get(c, "chol_flags", 8 * sizeof(int)));
  if (!W || !L || !flags) return PARO_ERR_CUDA;
  PARO_CU(c, cudaMemsetAsync(flags, 0, 8 * sizeof(int), c->stream));
  int grid = 1;
  int st = coop_grid(c, (const void*)k_chol, 256, 0, 64, &grid);
  if (st) return st;
  unsigned* bar = reinterpret_cast<unsigned*>(flags);
  int* err = flags + 2;
  int* info = flags + 3;
  cudaEvent_t ev = prof_begin(c);
  int nn = n;
  void* args[] = {&nn, (void*)&s, &W, &L, &g, &bar, &err, &info};
  PARO_CU(c, cudaLaunchCooperativeKernel((const void*)k_chol, dim3(grid), dim3(256), args, 0, c->stream));
  ++c->launches;
  prof_end(c, "k_chol", ev);
  int h[2] = {0, 0};
  PARO_CU(c, cudaMemcpyAsync(h, flags + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  if (h[0]) return fail(c, PARO_ERR_TIMEOUT, "Cholesky: grid barrier wait gave up");
  if (h[1]) return fail(c, PARO_ERR_BREAKDOWN, "Cholesky pivot <= 0 at column " + std::to_string(h[1] - 1));
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
  if constexpr (sizeof(T) == 4) {  // FP32 rows: FP32 squares (exact enough) in an FP32 two-sum pair
    float hi = 0.f, lo = 0.f;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) two_sum_acc(hi, lo, fmaf(xb[g].x, xb[g].x, xb[g].y * xb[g].y));
    acc = (double)hi + (double)lo;
  } else {
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
      const double re = xb[g].x, im = xb[g].y;
      acc += re * re + im * im;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[b] = acc;
}

// chunked form for long rows: partial sums per (band, chunk of 2048), then the chunks in order
template <typename T>
__global__ void k_band_norm2_part(int npw, const cplx<T>* __restrict__ x, int ldx, double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x, nch = gridDim.x;
  const cplx<T>* xb = x + (size_t)b * ldx;
  const int g0 = ch * 2048, g1 = min(npw, g0 + 2048);
  double acc = 0.0;
  if constexpr (sizeof(T) == 4) {
    float hi = 0.f, lo = 0.f;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) two_sum_acc(hi, lo, fmaf(xb[g].x, xb[g].x, xb[g].y * xb[g].y));
    acc = (double)hi + (double)lo;
  } else {
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      const double re = xb[g].x, im = xb[g].y;
      acc += re * re + im * im;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)b * nch + ch] = acc;
}

__global__ void k_band_norm2_sum(int nb, int nch, const double* __restrict__ part, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[(size_t)b * nch + ch];
  out[b] = s;
}

template <typename T>
int band_norms(Ctx* c, int nb, int npw, const cplx<T>* x, int ldx, double* out_dev) {
  const int nch = (npw + 2047) / 2048;
  if (nch <= 2) {
    k_band_norm2<T><<<nb, 256, 0, c->stream>>>(npw, x, ldx, out_dev);
    PARO_LAUNCH(c, "k_band_norm2");
    return PARO_OK;
  }
  double* part = static_cast<double*>(ws_get(c, "band_norm_part", (size_t)nb * nch * sizeof(double)));
  if (!part) return PARO_ERR_CUDA;
  k_band_norm2_part<T><<<dim3(nch, nb), 256, 0, c->stream>>>(npw, x, ldx, part);
  PARO_LAUNCH(c, "k_band_norm2_part");
  k_band_norm2_sum<<<(nb + 127) / 128, 128, 0, c->stream>>>(nb, nch, part, out_dev);
  PARO_LAUNCH(c, "k_band_norm2_sum");
  return PARO_OK;
}

// ||H psi_b - eps_b psi_b||. f32sq (mixed precision, whose orbitals carry FP32 rounding anyway): the
// difference in FP64 (it cancels), its square summed in an FP32 two-sum pair, a third of the FP64
// instructions and the norm to a relative 1e-7; otherwise all in FP64.
__global__ void k_resid(int npw, const double2* __restrict__ psi, const double2* __restrict__ hpsi,
                        const double* __restrict__ eps, double* __restrict__ out, int f32sq) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const double e = eps[b];
  double acc = 0.0;
  if (f32sq) {
    float hi = 0.f, lo = 0.f;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
      const double2 p = psi[(size_t)b * npw + g], h = hpsi[(size_t)b * npw + g];
      const float re = (float)fma(-e, p.x, h.x), im = (float)fma(-e, p.y, h.y);
      two_sum_acc(hi, lo, fmaf(re, re, im * im));
    }
    acc = (double)hi + (double)lo;
  } else {
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
      const double2 p = psi[(size_t)b * npw + g], h = hpsi[(size_t)b * npw + g];
      const double re = h.x - e * p.x, im = h.y - e * p.y;
      acc += re * re + im * im;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[b] = sqrt(acc);
}

// FP32 rows (mixed path): the row's chunk blockIdx.y of || h - eps p ||^2 with FP32 terms in an FP32
// two-sum pair; part[b * gridDim.y + chunk]. k_resid_final sums a band's chunks in order.
__global__ void __launch_bounds__(256) k_resid32(int npw, const float2* __restrict__ psi,
                                                 const float2* __restrict__ hpsi, const double* __restrict__ eps,
                                                 double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.x, len = (npw + gridDim.y - 1) / gridDim.y;
  const int g0 = blockIdx.y * len, g1 = min(npw, g0 + len);
  const float e = (float)eps[b];
  float hi = 0.f, lo = 0.f;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const float2 p = psi[(size_t)b * npw + g], h = hpsi[(size_t)b * npw + g];
    const float re = fmaf(-e, p.x, h.x), im = fmaf(-e, p.y, h.y);
    two_sum_acc(hi, lo, fmaf(re, re, im * im));
  }
  const double acc = block_sum((double)hi + (double)lo, red);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.y + blockIdx.y] = acc;
}

__global__ void k_resid_final(int nb, int nch, const double* __restrict__ part, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[(size_t)b * nch + ch];
  out[b] = sqrt(s);
}

int residual_norms32(Ctx* c, int nb, int npw, const float2* psi, const float2* hpsi, const double* eps_dev,
                     double* out_dev) {
  constexpr int kCh = 4;
  double* part = static_cast<double*>(ws_get(c, "resid_part", (size_t)nb * kCh * sizeof(double)));
  if (!part) return PARO_ERR_CUDA;
  k_resid32<<<dim3(nb, kCh), 256, 0, c->stream>>>(npw, psi, hpsi, eps_dev, part);
  PARO_LAUNCH(c, "k_resid32");
  k_resid_final<<<(nb + 127) / 128, 128, 0, c->stream>>>(nb, kCh, part, out_dev);
  PARO_LAUNCH(c, "k_resid_final");
  return PARO_OK;
}

int residual_norms(Ctx* c, int nb, int npw, const double2* psi, const double2* hpsi, const double* eps_dev,
                   double* out_dev) {
  k_resid<<<nb, 256, 0, c->stream>>>(npw, psi, hpsi, eps_dev, out_dev, c->prec == PARO_MIXED ? 1 : 0);
  PARO_LAUNCH(c, "k_resid");
  return PARO_OK;
}

// FP32 -> FP64 by the IEEE 754 bit layouts (sign, exponent rebiased by 1023 - 127, mantissa shifted by
// 29): exact, and on the integer pipe instead of GB300's narrow FP64 pipe; zeros, subnormals, infinities
// and NaNs take the ordinary conversion
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

template <typename TS, typename TD>
__global__ void k_convert(size_t n, const cplx<TS>* __restrict__ s, cplx<TD>* __restrict__ d) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(TS) == 4 && sizeof(TD) == 8)
      d[i] = mk<TD>(f32_to_f64_bits(s[i].x), f32_to_f64_bits(s[i].y));
    else
      d[i] = mk<TD>((TD)s[i].x, (TD)s[i].y);
  }
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
                                             int, bool, bool);
template int gemm_cn<float, float, float>(Ctx*, int, int, int, const float2*, int, const float2*, int, double2*, int,
                                          bool, bool);
template int gemm_wx<double, double>(Ctx*, int, int, int, const double2*, int, bool, const double*, const double2*,
                                     int, double2*, int, double, float2*, bool);
template int gemm_wx<float, float>(Ctx*, int, int, int, const double2*, int, bool, const double*, const float2*, int,
                                   float2*, int, double, float2*, bool);
template int gemm_wx<float, double>(Ctx*, int, int, int, const double2*, int, bool, const double*, const float2*,
                                    int, double2*, int, double, float2*, bool);
template int band_norms<double>(Ctx*, int, int, const double2*, int, double*);
template int band_norms<float>(Ctx*, int, int, const float2*, int, double*);
template int convert<double, float>(Ctx*, size_t, const double2*, float2*);
template int convert<float, double>(Ctx*, size_t, const float2*, double2*);

}  // namespace paro
