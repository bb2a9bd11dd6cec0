// Complex FP32 products on the tensor cores (tcgen05, kind::tf32) with the 3xTF32 split: every FP32
// operand x = hi + lo (hi, lo TF32), a b ~ ah bh + ah bl + al bh accumulated in FP32 in tensor memory;
// the dropped al bl and the rounding of lo keep the product within a few FP32 ulps.
//
// Complex arithmetic as real products on the interleaved storage: a row of complex values
// (re0, im0, re1, im1, ...) is a real row of twice the length, so for C = conj(A) B^T
//   Re C = A' . B'              (A', B' the interleaved rows)
//   Im C = A'' . B',  A'' = (-im0, re0, -im1, re1, ...)
// A'' is formed in registers while the tile is staged. Two accumulators per tile (Re in TMEM columns
// 0.., Im in 256..), six MMAs per 8-wide K step.
//
// Staging: threads load the tile rows from global memory (8-byte loads: rows of odd length are not
// 16-byte aligned), split them, and store them in the no-swizzle K-major core-matrix layout (8 rows x
// 16 bytes contiguous); one thread issues the MMAs and commits them to an mbarrier that every thread
// waits on (bounded) before the next stage overwrites the tile.
#include <algorithm>

#include "paro_ctx.h"
#include "tc_sm100.cuh"

namespace paro {

static const int kTcM = 128;       // rows of A per CTA = TMEM lanes
static const int kTcKc = 16;       // complex K elements per stage (32 reals = 4 MMAs of 8)
static const int kTcCh = kTcKc * 2 * 4 / 16;  // 16-byte chunks per row per stage (8)
static const int kTcThreads = 256;
static const uint32_t kTcPolls = 1u << 24;

__device__ __forceinline__ uint32_t tc_off(int row, int chunk) {
  return (uint32_t)(((row >> 3) * kTcCh + chunk) * 128 + (row & 7) * 16);
}

// split (v0, v1) into hi and lo TF32 quadruples (re0, im0, re1, im1)
__device__ __forceinline__ void tc_split(float2 v0, float2 v1, float4& h, float4& l) {
  h.x = tc::tf32_round(v0.x); h.y = tc::tf32_round(v0.y); h.z = tc::tf32_round(v1.x); h.w = tc::tf32_round(v1.y);
  l.x = tc::tf32_round(v0.x - h.x); l.y = tc::tf32_round(v0.y - h.y);
  l.z = tc::tf32_round(v1.x - h.z); l.w = tc::tf32_round(v1.y - h.w);
}

// part[z][m][n] = sum over K slice z of conj(A[m][k]) B[n][k] (complex double). NT: N tile (multiple of
// 16, at most 256). err: set when an mbarrier wait gives up.
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_cn_tc(int M, int N, int K, int kslice, int NT,
                                                              const float2* __restrict__ A, int lda,
                                                              const float2* __restrict__ B, int ldb,
                                                              double2* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int A_BYTES = kTcM * kTcCh * 16, B_BYTES = NT * kTcCh * 16;
  unsigned char* sAh = smem;
  unsigned char* sAl = smem + A_BYTES;
  unsigned char* sAph = smem + 2 * A_BYTES;
  unsigned char* sApl = smem + 3 * A_BYTES;
  unsigned char* sBh = smem + 4 * A_BYTES;
  unsigned char* sBl = sBh + B_BYTES;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * NT;
  const int k0 = blockIdx.z * kslice, k1 = min(K, k0 + kslice);
  const uint32_t ncols = NT <= 128 ? 256u : 512u;  // Re and Im accumulators, NT columns each
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t dR = tmem_base, dI = tmem_base + ncols / 2;
  const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)NT);
  const uint32_t aH = tc::smem_addr(sAh), aL = tc::smem_addr(sAl), apH = tc::smem_addr(sAph),
                 apL = tc::smem_addr(sApl), bH = tc::smem_addr(sBh), bL = tc::smem_addr(sBl);
  uint32_t phase = 0;
  int ok = 1, nst = 0;
  for (int kk = k0; kk < k1; kk += kTcKc, ++nst) {
    for (int i = tid; i < kTcM * kTcCh; i += kTcThreads) {
      const int r = i / kTcCh, ch = i - r * kTcCh;
      const int gm = m0 + r, g0 = kk + 2 * ch;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (gm < M) {
        const float2* row = A + (size_t)gm * lda;
        if (g0 < k1) v0 = row[g0];
        if (g0 + 1 < k1) v1 = row[g0 + 1];
      }
      float4 h, l;
      tc_split(v0, v1, h, l);
      const uint32_t o = tc_off(r, ch);
      *reinterpret_cast<float4*>(sAh + o) = h;
      *reinterpret_cast<float4*>(sAl + o) = l;
      *reinterpret_cast<float4*>(sAph + o) = make_float4(-h.y, h.x, -h.w, h.z);
      *reinterpret_cast<float4*>(sApl + o) = make_float4(-l.y, l.x, -l.w, l.z);
    }
    for (int i = tid; i < NT * kTcCh; i += kTcThreads) {
      const int r = i / kTcCh, ch = i - r * kTcCh;
      const int gn = n0 + r, g0 = kk + 2 * ch;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (gn < N) {
        const float2* row = B + (size_t)gn * ldb;
        if (g0 < k1) v0 = row[g0];
        if (g0 + 1 < k1) v1 = row[g0 + 1];
      }
      float4 h, l;
      tc_split(v0, v1, h, l);
      const uint32_t o = tc_off(r, ch);
      *reinterpret_cast<float4*>(sBh + o) = h;
      *reinterpret_cast<float4*>(sBl + o) = l;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int s = 0; s < kTcCh / 2; ++s) {
        const uint32_t off = (uint32_t)s * 256u;  // two 16-byte chunks (8 TF32) per MMA
        const uint32_t lbo = 128u, sbo = kTcCh * 128u;
        const uint64_t dAh = tc::smem_desc(aH + off, lbo, sbo), dAl = tc::smem_desc(aL + off, lbo, sbo);
        const uint64_t dApH = tc::smem_desc(apH + off, lbo, sbo), dApL = tc::smem_desc(apL + off, lbo, sbo);
        const uint64_t dBh = tc::smem_desc(bH + off, lbo, sbo), dBl = tc::smem_desc(bL + off, lbo, sbo);
        const uint32_t acc = (nst > 0 || s > 0) ? 1u : 0u;
        tc::mma_tf32(dR, dAh, dBh, idesc, acc);
        tc::mma_tf32(dR, dAh, dBl, idesc, 1u);
        tc::mma_tf32(dR, dAl, dBh, idesc, 1u);
        tc::mma_tf32(dI, dApH, dBh, idesc, acc);
        tc::mma_tf32(dI, dApH, dBl, idesc, 1u);
        tc::mma_tf32(dI, dApL, dBh, idesc, 1u);
      }
      tc::mma_commit(&mbar);
    }
    const int done = tc::mbar_wait(&mbar, phase, kTcPolls) ? 1 : 0;
    ok = __syncthreads_and(done);
    if (!ok) {  // give the MMAs in flight one more bounded wait before tensor memory is released
      tc::mbar_wait(&mbar, phase, kTcPolls);
      break;
    }
    phase ^= 1u;
  }
  tc::tc_fence_after();
  // accumulators: warp w reads TMEM lanes 32 (w % 4) ..; warps w and w + 4 split the columns
  const int lq = warp & 3, half = warp >> 2;
  const int row = m0 + 32 * lq + lane;
  const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
  double2* pz = part + (size_t)blockIdx.z * M * N;
  for (int cb = 8 * half; cb < NT; cb += 16) {
    float re[8], im[8];
    tc::tmem_ld_x8(dR + lane_off + (uint32_t)cb, re);
    tc::tmem_ld_x8(dI + lane_off + (uint32_t)cb, im);
    if (row < M) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n0 + cb + j;
        if (n < N)
          pz[(size_t)row * N + n] = (ok && nst > 0) ? make_double2((double)re[j], (double)im[j]) : make_double2(0.0, 0.0);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, ncols);
  }
  if (!ok && tid == 0) atomicExch(err, 1);
}

// Y[m][n] = beta Y[m][n] + sum_k s_k W(k, m) X[k][n] (complex FP32 X, Y; complex double W, W(k, m) at
// W[k ldw + m], or W[m ldw + k] when wt; s: per-k scale or null). The MMA tile is D[n][m] = sum_k A[n][k]
// B[m][k] with A = X^T (the long N_pw dimension on the 128 TMEM lanes, transposed while staged) and
// B[m][k] = s_k W(k, m):  Re D = A' . (Br, -Bi)',  Im D = A' . (Bi, Br)'  on the interleaved rows.
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_wx_tc(int M, int N, int K, int NT,
                                                              const double2* __restrict__ W, int ldw, int wt,
                                                              const double* __restrict__ sc,
                                                              const float2* __restrict__ X, int ldx,
                                                              float2* __restrict__ Y, int ldy, float beta,
                                                              int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int A_BYTES = kTcM * kTcCh * 16, B_BYTES = NT * kTcCh * 16;
  unsigned char* sAh = smem;
  unsigned char* sAl = smem + A_BYTES;
  unsigned char* sRh = smem + 2 * A_BYTES;  // B for Re: (Br, -Bi)
  unsigned char* sRl = sRh + B_BYTES;
  unsigned char* sIh = sRl + B_BYTES;       // B for Im: (Bi, Br)
  unsigned char* sIl = sIh + B_BYTES;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kTcM, m0 = blockIdx.y * NT;
  const uint32_t ncols = NT <= 128 ? 256u : 512u;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t dR = tmem_base, dI = tmem_base + ncols / 2;
  const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)NT);
  const uint32_t aH = tc::smem_addr(sAh), aL = tc::smem_addr(sAl), rH = tc::smem_addr(sRh), rL = tc::smem_addr(sRl),
                 iH = tc::smem_addr(sIh), iL = tc::smem_addr(sIl);
  uint32_t phase = 0;
  int ok = 1, nst = 0;
  for (int kk = 0; kk < K; kk += kTcKc, ++nst) {
    for (int i = tid; i < kTcM * kTcCh; i += kTcThreads) {  // consecutive threads: consecutive n (rows)
      const int r = i % kTcM, ch = i / kTcM;
      const int gn = n0 + r, k0 = kk + 2 * ch;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (gn < N) {
        if (k0 < K) v0 = X[(size_t)k0 * ldx + gn];
        if (k0 + 1 < K) v1 = X[(size_t)(k0 + 1) * ldx + gn];
      }
      float4 h, l;
      tc_split(v0, v1, h, l);
      const uint32_t o = tc_off(r, ch);
      *reinterpret_cast<float4*>(sAh + o) = h;
      *reinterpret_cast<float4*>(sAl + o) = l;
    }
    for (int i = tid; i < NT * kTcCh; i += kTcThreads) {
      const int r = i / kTcCh, ch = i - r * kTcCh;
      const int gm = m0 + r, k0 = kk + 2 * ch;
      float2 b0 = make_float2(0.f, 0.f), b1 = b0;
      if (gm < M) {
        if (k0 < K) {
          const double2 w = wt ? W[(size_t)gm * ldw + k0] : W[(size_t)k0 * ldw + gm];
          const double f = sc ? sc[k0] : 1.0;
          b0 = make_float2((float)(f * w.x), (float)(f * w.y));
        }
        if (k0 + 1 < K) {
          const double2 w = wt ? W[(size_t)gm * ldw + k0 + 1] : W[(size_t)(k0 + 1) * ldw + gm];
          const double f = sc ? sc[k0 + 1] : 1.0;
          b1 = make_float2((float)(f * w.x), (float)(f * w.y));
        }
      }
      float4 h, l;
      tc_split(b0, b1, h, l);
      const uint32_t o = tc_off(r, ch);
      *reinterpret_cast<float4*>(sRh + o) = make_float4(h.x, -h.y, h.z, -h.w);
      *reinterpret_cast<float4*>(sRl + o) = make_float4(l.x, -l.y, l.z, -l.w);
      *reinterpret_cast<float4*>(sIh + o) = make_float4(h.y, h.x, h.w, h.z);
      *reinterpret_cast<float4*>(sIl + o) = make_float4(l.y, l.x, l.w, l.z);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int s = 0; s < kTcCh / 2; ++s) {
        const uint32_t off = (uint32_t)s * 256u;
        const uint32_t lbo = 128u, sbo = kTcCh * 128u;
        const uint64_t dAh = tc::smem_desc(aH + off, lbo, sbo), dAl = tc::smem_desc(aL + off, lbo, sbo);
        const uint64_t dRh = tc::smem_desc(rH + off, lbo, sbo), dRl = tc::smem_desc(rL + off, lbo, sbo);
        const uint64_t dIh = tc::smem_desc(iH + off, lbo, sbo), dIl = tc::smem_desc(iL + off, lbo, sbo);
        const uint32_t acc = (nst > 0 || s > 0) ? 1u : 0u;
        tc::mma_tf32(dR, dAh, dRh, idesc, acc);
        tc::mma_tf32(dR, dAh, dRl, idesc, 1u);
        tc::mma_tf32(dR, dAl, dRh, idesc, 1u);
        tc::mma_tf32(dI, dAh, dIh, idesc, acc);
        tc::mma_tf32(dI, dAh, dIl, idesc, 1u);
        tc::mma_tf32(dI, dAl, dIh, idesc, 1u);
      }
      tc::mma_commit(&mbar);
    }
    const int done = tc::mbar_wait(&mbar, phase, kTcPolls) ? 1 : 0;
    ok = __syncthreads_and(done);
    if (!ok) {
      tc::mbar_wait(&mbar, phase, kTcPolls);
      break;
    }
    phase ^= 1u;
  }
  tc::tc_fence_after();
  const int lq = warp & 3, half = warp >> 2;
  const int gn = n0 + 32 * lq + lane;
  const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
  for (int cb = 8 * half; cb < NT; cb += 16) {
    float re[8], im[8];
    tc::tmem_ld_x8(dR + lane_off + (uint32_t)cb, re);
    tc::tmem_ld_x8(dI + lane_off + (uint32_t)cb, im);
    if (gn < N) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int m = m0 + cb + j;
        if (m < M) {
          float2* y = Y + (size_t)m * ldy + gn;
          const float vr = (ok && nst > 0) ? re[j] : 0.f, vi = (ok && nst > 0) ? im[j] : 0.f;
          if (beta != 0.f) {
            const float2 o = *y;
            *y = make_float2(beta * o.x + vr, beta * o.y + vi);
          } else {
            *y = make_float2(vr, vi);
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, ncols);
  }
  if (!ok && tid == 0) atomicExch(err, 1);
}

static size_t tc_smem_wx(int NT) { return (size_t)2 * kTcM * kTcCh * 16 + (size_t)4 * NT * kTcCh * 16; }

int gemm_wx_tc(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s, const float2* X,
               int ldx, float2* Y, int ldy, double beta, int* err) {
  const int mtiles = (M + 255) / 256;
  const int nt = ((M + mtiles - 1) / mtiles + 15) / 16 * 16;
  static int attr_dev = -1;
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (attr_dev != dev) {
    PARO_CU(c, cudaFuncSetAttribute(k_gemm_wx_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_wx(256)));
    attr_dev = dev;
  }
  k_gemm_wx_tc<<<dim3((N + kTcM - 1) / kTcM, mtiles), kTcThreads, tc_smem_wx(nt), c->stream>>>(
      M, N, K, nt, W, ldw, wt ? 1 : 0, s, X, ldx, Y, ldy, (float)beta, err);
  PARO_LAUNCH(c, "k_gemm_wx_tc");
  return PARO_OK;
}

static size_t tc_smem(int NT) { return (size_t)4 * kTcM * kTcCh * 16 + (size_t)2 * NT * kTcCh * 16; }

// K split of the tensor-core product: one CTA per SM, the slice count minimising waves x stages per
// slice (at least 4 stages per slice), and no slice longer than 8192 complex terms, so the FP32 sum in
// tensor memory stays short (slices are added in FP64).
void gemm_cn_tc_plan(int M, int N, int K, int* nz_out, int* kslice_out) {
  const int ntiles = (N + 255) / 256;
  const int mtiles = (M + kTcM - 1) / kTcM;
  const int tiles = mtiles * ntiles;
  const int steps = (K + kTcKc - 1) / kTcKc;
  const int maxz = std::max(1, steps / 4);
  const int minz = (steps + 8192 / kTcKc - 1) / (8192 / kTcKc);
  int best_nz = minz;
  long long best = -1;
  for (int z = std::min(minz, maxz); z <= std::min(std::max(maxz, minz), 1024); ++z) {
    const int s = (steps + z - 1) / z;
    const int zz = (steps + s - 1) / s;
    const long long cost = (long long)((tiles * zz + 151) / 152) * s;
    if (best < 0 || cost < best) {
      best = cost;
      best_nz = zz;
    }
  }
  const int kslice = ((steps + best_nz - 1) / best_nz) * kTcKc;
  *kslice_out = kslice;
  *nz_out = std::max(1, (K + kslice - 1) / kslice);
}

// Tensor-core path of gemm_cn<float, float, float> (no Hermitian half, no carry): the same partial-sum
// layout as the CUDA-core kernel, reduced by k_reduce_parts; part holds nz x M x N (gemm_cn_tc_plan).
int gemm_cn_tc(Ctx* c, int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, double2* part,
               int kslice, int nz, int* err) {
  const int ntiles = (N + 255) / 256;
  const int nt = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
  const int mtiles = (M + kTcM - 1) / kTcM;
  static int attr_dev = -1;
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (attr_dev != dev) {
    PARO_CU(c, cudaFuncSetAttribute(k_gemm_cn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(256)));
    attr_dev = dev;
  }
  k_gemm_cn_tc<<<dim3(mtiles, ntiles, nz), kTcThreads, tc_smem(nt), c->stream>>>(M, N, K, kslice, nt, A, lda, B, ldb,
                                                                                 part, err);
  PARO_LAUNCH(c, "k_gemm_cn_tc");
  return PARO_OK;
}

}  // namespace paro
