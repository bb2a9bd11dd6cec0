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
static const int kTcThreads = 256;
static const uint32_t kTcPolls = 1u << 24;

// Pipeline of the tensor-core kernels: two shared-memory buffers, one mbarrier each. Stage s is staged into
// buffer s & 1 while the MMAs of stage s - 1 run on the other; before a buffer is overwritten, the MMAs of
// stage s - 2 (its previous use) must have completed. Every wait is bounded; on a time-out the kernel
// waits once more for the MMAs in flight, reports, and still releases tensor memory.
struct TcPipe {
  uint64_t* bar;      // [2]
  uint32_t uses[2];   // completed uses waited for, per buffer
  int ok;
  const int* fail;    // shared flag set by the MMA-issuing thread (its own copy wait gave up), or null
  __device__ __forceinline__ bool wait_buffer(int b) {  // all threads; uniform result
    const int done = tc::mbar_wait(&bar[b], uses[b] & 1u, kTcPolls) ? 1 : 0;
    ok = __syncthreads_and(done && ok && !(fail && *fail));
    if (ok) ++uses[b];
    return ok;
  }
};

// part[z][m][n] = sum over K slice z of conj(A[m][k]) B[n][k] (complex, FP32 as the tensor memory holds
// it). NT: N tile (multiple of 16, at most 256). Stages of KC = 8 complex K values. err: set when an
// mbarrier wait gives up.
//
// Pipeline: NR raw stages of plain FP32 rows (A rows m0.., then B rows n0..; 80-byte row pitch so that the
// split's 16-byte reads are conflict-free) are filled by cp.async NR - 1 stages ahead; each iteration splits
// one raw stage into the six operand tiles of one of two operand buffers (hi, lo of A' and A'', hi, lo of
// B') while the MMAs of the previous stage run, then one thread issues the stage's 12 MMAs.
static const int kCnKC = 8, kCnCh = 4, kRawPitch = 80;
template <int NR>
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_cn_tc(int M, int N, int K, int kslice, int NT,
                                                              const float2* __restrict__ A, int lda,
                                                              const float2* __restrict__ B, int ldb,
                                                              float2* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = tc_align1024(smem_dyn);
  constexpr int ch = kCnCh;
  const int A_BYTES = kTcM * ch * 16, B_BYTES = NT * ch * 16, STAGE = 4 * A_BYTES + 2 * B_BYTES;
  const int RROWS = kTcM + NT, RAW = RROWS * kRawPitch;
  unsigned char* raw0 = smem + 2 * STAGE;
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * NT;
  const int k0 = blockIdx.z * kslice, k1 = min(K, k0 + kslice);
  const int nst = k1 > k0 ? (k1 - k0 + kCnKC - 1) / kCnKC : 0;
  const uint32_t ncols = NT <= 128 ? 256u : 512u;  // Re and Im accumulators, NT columns each
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t dR = tmem_base, dI = tmem_base + ncols / 2;
  const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)NT);
  // raw stage s: row r (A rows, then B rows) x 8 complex; one 8-byte copy per element, zero-filled outside
  auto issue = [&](int st) {
    unsigned char* raw = raw0 + (st % NR) * RAW;
    const int kk = k0 + st * kCnKC;
    for (int i = tid; i < RROWS * kCnKC; i += kTcThreads) {
      const int r = i >> 3, kx = i & 7, gk = kk + kx;
      const float2* src;
      bool in;
      if (r < kTcM) {
        in = m0 + r < M && gk < k1;
        src = in ? A + (size_t)(m0 + r) * lda + gk : A;
      } else {
        in = n0 + r - kTcM < N && gk < k1;
        src = in ? B + (size_t)(n0 + r - kTcM) * ldb + gk : B;
      }
      cp_async8(raw + r * kRawPitch + kx * 8, src, in ? 8 : 0);
    }
  };
  TcPipe pipe{mbar, {0u, 0u}, 1, nullptr};
  int issued[2] = {0, 0};
#pragma unroll
  for (int p = 0; p < NR - 1; ++p) {
    if (p < nst) issue(p);
    cp_async_commit();
  }
  int s = 0;
  for (; s < nst; ++s) {
    if (s + NR - 1 < nst) issue(s + NR - 1);  // into the slot read in iteration s - 1 (past its barrier)
    cp_async_commit();
    cp_async_wait<NR - 1>();  // this thread's copies of raw stage s have landed
    const int b = s & 1;
    if (issued[b]) {
      if (!pipe.wait_buffer(b)) break;  // barrier: raw stage s visible, operand buffer b free
    } else {
      __syncthreads();
    }
    issued[b] = 0;
    unsigned char* sAh = smem + b * STAGE;
    unsigned char* sAl = sAh + A_BYTES;
    unsigned char* sAph = sAl + A_BYTES;
    unsigned char* sApl = sAph + A_BYTES;
    unsigned char* sBh = sApl + A_BYTES;
    unsigned char* sBl = sBh + B_BYTES;
    const unsigned char* raw = raw0 + (s % NR) * RAW;
    // unit i -> (row, chunk): 8 consecutive threads take the 8 rows of one core matrix at one chunk
    for (int i = tid; i < kTcM * ch; i += kTcThreads) {
      const int r = (i & 7) + 8 * (i / (8 * ch)), c = (i >> 3) % ch;
      const float4 v = *reinterpret_cast<const float4*>(raw + r * kRawPitch + c * 16);
      float4 h, l;
      tc_split(make_float2(v.x, v.y), make_float2(v.z, v.w), h, l);
      const uint32_t o = tc_off(r, c, ch);
      *reinterpret_cast<float4*>(sAh + o) = h;
      *reinterpret_cast<float4*>(sAl + o) = l;
      *reinterpret_cast<float4*>(sAph + o) = make_float4(-h.y, h.x, -h.w, h.z);
      *reinterpret_cast<float4*>(sApl + o) = make_float4(-l.y, l.x, -l.w, l.z);
    }
    for (int i = tid; i < NT * ch; i += kTcThreads) {
      const int r = (i & 7) + 8 * (i / (8 * ch)), c = (i >> 3) % ch;
      const float4 v = *reinterpret_cast<const float4*>(raw + (kTcM + r) * kRawPitch + c * 16);
      float4 h, l;
      tc_split(make_float2(v.x, v.y), make_float2(v.z, v.w), h, l);
      const uint32_t o = tc_off(r, c, ch);
      *reinterpret_cast<float4*>(sBh + o) = h;
      *reinterpret_cast<float4*>(sBl + o) = l;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t aH = tc::smem_addr(sAh), aL = tc::smem_addr(sAl), apH = tc::smem_addr(sAph),
                     apL = tc::smem_addr(sApl), bH = tc::smem_addr(sBh), bL = tc::smem_addr(sBl);
      for (int s2 = 0; s2 < ch / 2; ++s2) {  // two 16-byte chunks (8 TF32) per MMA
        const uint64_t dAh = tc_desc(aH, s2, ch), dAl = tc_desc(aL, s2, ch);
        const uint64_t dApH = tc_desc(apH, s2, ch), dApL = tc_desc(apL, s2, ch);
        const uint64_t dBh = tc_desc(bH, s2, ch), dBl = tc_desc(bL, s2, ch);
        const uint32_t acc = (s > 0 || s2 > 0) ? 1u : 0u;
        tc::mma_tf32(dR, dAh, dBh, idesc, acc);
        tc::mma_tf32(dR, dAh, dBl, idesc, 1u);
        tc::mma_tf32(dR, dAl, dBh, idesc, 1u);
        tc::mma_tf32(dI, dApH, dBh, idesc, acc);
        tc::mma_tf32(dI, dApH, dBl, idesc, 1u);
        tc::mma_tf32(dI, dApL, dBh, idesc, 1u);
      }
      tc::mma_commit(&mbar[b]);
    }
    issued[b] = 1;
  }
  cp_async_wait<0>();  // no copy into shared memory outlives the CTA
  // drain: the last one or two stages
  for (int b = 0; b < 2; ++b)
    if (issued[b] && pipe.ok && !pipe.wait_buffer(b)) break;
  if (!pipe.ok) {  // one more bounded wait for MMAs in flight before tensor memory is released
    for (int b = 0; b < 2; ++b)
      if (issued[b]) tc::mbar_wait(&mbar[b], pipe.uses[b] & 1u, kTcPolls);
  }
  const int ok = pipe.ok;
  tc::tc_fence_after();
  // accumulators: warp w reads TMEM lanes 32 (w % 4) ..; warps w and w + 4 split the columns
  const int lq = warp & 3, half = warp >> 2;
  const int row = m0 + 32 * lq + lane;
  const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
  float2* pz = part + (size_t)blockIdx.z * M * N;
  const bool have = ok && nst > 0;
  for (int cb = 8 * half; cb < NT; cb += 16) {
    float re[8], im[8];
    tc::tmem_ld_x8(dR + lane_off + (uint32_t)cb, re);
    tc::tmem_ld_x8(dI + lane_off + (uint32_t)cb, im);
    if (row < M) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n0 + cb + j;
        if (n < N) pz[(size_t)row * N + n] = have ? make_float2(re[j], im[j]) : make_float2(0.f, 0.f);
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

// C[m][n] = sum over z of part[z][m][n] in a fixed order, added into an FP32 two-sum pair (no FP64 pipe)
__global__ void k_reduce_parts32(int M, int N, int nz, const float2* __restrict__ part, double2* __restrict__ C,
                                 int ldc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
  for (int z = 0; z < nz; ++z) {
    const float2 v = part[(size_t)z * M * N + idx];
    two_sum_acc(hx, lx, v.x);
    two_sum_acc(hy, ly, v.y);
  }
  const int m = idx / N, n = idx - m * N;
  C[(size_t)m * ldc + n] = make_double2((double)hx + (double)lx, (double)hy + (double)ly);
}

// Y[m][n] = beta Y[m][n] + sum_k s_k W(k, m) X[k][n] (complex FP32 X, Y; complex double W, W(k, m) at
// W[k ldw + m], or W[m ldw + k] when wt; s: per-k scale or null). The MMA tile is D[n][m] = sum_k A[n][k]
// B[m][k] with A = X^T (the long N_pw dimension on the 128 TMEM lanes, transposed while staged) and
// B[m][k] = s_k W(k, m):  Re D = A' . (Br, -Bi)',  Im D = A' . (Bi, Br)'  on the interleaved rows.
// The four B tiles of every stage are split once per call by k_wx_presplit (Wp) and copied with 16-byte
// loads.
__global__ void k_wx_presplit(int M, int K, int NT, int KC, const double2* __restrict__ W, int ldw, int wt,
                              const double* __restrict__ sc, float4* __restrict__ Wp) {
  const int ch = KC / 2, nstage = (K + KC - 1) / KC;
  const int mt = blockIdx.y;  // M tile
  const size_t tile = (size_t)NT * ch;  // float4 per variant per stage
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)nstage * tile;
       i += (size_t)gridDim.x * blockDim.x) {
    const int st = (int)(i / tile);
    const int rem = (int)(i - (size_t)st * tile);
    const int r = rem / ch, c = rem - r * ch;
    const int gm = mt * NT + r, k0 = st * KC + 2 * c;
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
    const size_t base = (((size_t)mt * nstage + st) * 4) * tile;
    const uint32_t o = tc_off(r, c, ch) / 16;  // float4 index within a variant tile
    Wp[base + 0 * tile + o] = make_float4(h.x, -h.y, h.z, -h.w);  // Re, hi
    Wp[base + 1 * tile + o] = make_float4(l.x, -l.y, l.z, -l.w);  // Re, lo
    Wp[base + 2 * tile + o] = make_float4(h.y, h.x, h.w, h.z);    // Im, hi
    Wp[base + 3 * tile + o] = make_float4(l.y, l.x, l.w, l.z);    // Im, lo
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_wx_tc(int M, int N, int K, int NT, int KC,
                                                              const float4* __restrict__ Wp,
                                                              const float2* __restrict__ X, int ldx,
                                                              float2* __restrict__ Y, int ldy, float beta,
                                                              int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = tc_align1024(smem_dyn);
  const int ch = KC / 2, nstage = (K + KC - 1) / KC;
  const int A_BYTES = kTcM * ch * 16, B_BYTES = NT * ch * 16, STAGE = 2 * A_BYTES + 4 * B_BYTES;
  __shared__ uint64_t mbar[2], fbar[2];  // MMAs done / B tiles landed, per buffer
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kTcM, mt = blockIdx.y, m0 = mt * NT;
  const uint32_t ncols = NT <= 128 ? 256u : 512u;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init(&fbar[0], 1);
    tc::mbar_init(&fbar[1], 1);
    s_fail = 0;
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t dR = tmem_base, dI = tmem_base + ncols / 2;
  const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)NT);
  const size_t tile4 = (size_t)NT * ch;  // float4 per B variant per stage
  TcPipe pipe{mbar, {0u, 0u}, 1, &s_fail};
  int issued[2] = {0, 0};
  uint32_t fuses[2] = {0u, 0u};  // thread 0: completed phases of fbar
  int pend[2] = {0, 0};           // thread 0: a bulk copy into this buffer not yet seen complete
  const uint32_t bbytes = (uint32_t)(4 * B_BYTES);
  int nst = 0;
  for (; nst < nstage; ++nst) {
    const int b = nst & 1, kk = nst * KC;
    if (issued[b] && !pipe.wait_buffer(b)) break;
    issued[b] = 0;
    unsigned char* sAh = smem + b * STAGE;
    unsigned char* sAl = sAh + A_BYTES;
    unsigned char* sB = sAl + A_BYTES;  // 4 variant tiles: Re hi, Re lo, Im hi, Im lo
    if (tid == 0) {  // the presplit B tiles of this stage: one bulk copy (contiguous in Wp)
      tc::mbar_arrive_expect_tx(&fbar[b], bbytes);
      tc::bulk_g2s(sB, Wp + (((size_t)mt * nstage + nst) * 4) * tile4, bbytes, &fbar[b]);
      pend[b] = 1;
    }
    {  // consecutive threads: consecutive n (rows); all loads before any split or store
      constexpr int UA = kTcM * 8 / kTcThreads;
      float2 va[UA][2];
#pragma unroll
      for (int t = 0; t < UA; ++t) {
        const int i = tid + t * kTcThreads;
        va[t][0] = va[t][1] = make_float2(0.f, 0.f);
        if (i < kTcM * ch) {
          const int r = i % kTcM, c = i / kTcM;
          const int gn = n0 + r, k0 = kk + 2 * c;
          if (gn < N) {
            if (k0 < K) va[t][0] = X[(size_t)k0 * ldx + gn];
            if (k0 + 1 < K) va[t][1] = X[(size_t)(k0 + 1) * ldx + gn];
          }
        }
      }
#pragma unroll
      for (int t = 0; t < UA; ++t) {
        const int i = tid + t * kTcThreads;
        if (i >= kTcM * ch) continue;
        const int r = i % kTcM, c = i / kTcM;
        float4 h, l;
        tc_split(va[t][0], va[t][1], h, l);
        const uint32_t o = tc_off(r, c, ch);
        *reinterpret_cast<float4*>(sAh + o) = h;
        *reinterpret_cast<float4*>(sAl + o) = l;
      }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      const bool landed = tc::mbar_wait(&fbar[b], fuses[b] & 1u, kTcPolls);
      if (landed) {
        ++fuses[b];
        pend[b] = 0;
      } else {
        s_fail = 1;  // no MMAs for this stage; the commit below still arrives
      }
      tc::tc_fence_after();
      const uint32_t aH = tc::smem_addr(sAh), aL = tc::smem_addr(sAl), bb = tc::smem_addr(sB);
      const uint32_t rH = bb, rL = bb + B_BYTES, iH = bb + 2 * B_BYTES, iL = bb + 3 * B_BYTES;
      for (int s2 = 0; landed && s2 < ch / 2; ++s2) {
        const uint64_t dAh = tc_desc(aH, s2, ch), dAl = tc_desc(aL, s2, ch);
        const uint64_t dRh = tc_desc(rH, s2, ch), dRl = tc_desc(rL, s2, ch);
        const uint64_t dIh = tc_desc(iH, s2, ch), dIl = tc_desc(iL, s2, ch);
        const uint32_t acc = (nst > 0 || s2 > 0) ? 1u : 0u;
        tc::mma_tf32(dR, dAh, dRh, idesc, acc);
        tc::mma_tf32(dR, dAh, dRl, idesc, 1u);
        tc::mma_tf32(dR, dAl, dRh, idesc, 1u);
        tc::mma_tf32(dI, dAh, dIh, idesc, acc);
        tc::mma_tf32(dI, dAh, dIl, idesc, 1u);
        tc::mma_tf32(dI, dAl, dIh, idesc, 1u);
      }
      tc::mma_commit(&mbar[b]);
    }
    issued[b] = 1;
  }
  for (int b = 0; b < 2; ++b)
    if (issued[b] && pipe.ok && !pipe.wait_buffer(b)) break;
  if (!pipe.ok) {
    for (int b = 0; b < 2; ++b)
      if (issued[b]) tc::mbar_wait(&mbar[b], pipe.uses[b] & 1u, kTcPolls);
  }
  if (tid == 0)  // a bulk copy still in flight after a time-out lands before the CTA leaves
    for (int b = 0; b < 2; ++b)
      if (pend[b]) tc::mbar_wait(&fbar[b], fuses[b] & 1u, kTcPolls);
  const int ok = pipe.ok;
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

// dynamic shared memory of the two-buffer pipelines; KC = 16 complex per stage where both buffers fit,
// else 8
static size_t wx_stage_bytes(int NT, int KC) { return (size_t)(2 * kTcM + 4 * NT) * (KC / 2) * 16; }
static const size_t kTcSmemMax = 220 * 1024;
static const size_t kTcAlignPad = 1024;  // room to align the stage buffers to 1024 bytes
static int wx_kc(int NT) { return 2 * wx_stage_bytes(NT, 16) + kTcAlignPad <= kTcSmemMax ? 16 : 8; }

static int set_smem_attr(Ctx* c, const void* k, int* dev_done) {
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (*dev_done != dev) {
    PARO_CU(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax));
    *dev_done = dev;
  }
  return PARO_OK;
}

int gemm_wx_tc(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s, const float2* X,
               int ldx, float2* Y, int ldy, double beta, int* err) {
  const int mtiles = (M + 255) / 256;
  const int nt = ((M + mtiles - 1) / mtiles + 15) / 16 * 16;
  const int kc = wx_kc(nt);
  const int nstage = std::max(1, (K + kc - 1) / kc);
  const size_t tile4 = (size_t)nt * (kc / 2);
  float4* Wp = static_cast<float4*>(ws_get(c, "tc_wx_split", (size_t)mtiles * nstage * 4 * tile4 * sizeof(float4)));
  if (!Wp) return PARO_ERR_CUDA;
  static int attr_dev = -1;
  int st;
  if ((st = set_smem_attr(c, (const void*)k_gemm_wx_tc, &attr_dev))) return st;
  if (K > 0) {
    k_wx_presplit<<<dim3(64, mtiles), 256, 0, c->stream>>>(M, K, nt, kc, W, ldw, wt ? 1 : 0, s, Wp);
    PARO_LAUNCH(c, "k_wx_presplit");
  }
  k_gemm_wx_tc<<<dim3((N + kTcM - 1) / kTcM, mtiles), kTcThreads, 2 * wx_stage_bytes(nt, kc) + kTcAlignPad, c->stream>>>(
      M, N, K, nt, kc, Wp, X, ldx, Y, ldy, (float)beta, err);
  PARO_LAUNCH(c, "k_gemm_wx_tc");
  return PARO_OK;
}

// shared memory of the projection pipeline: two operand buffers, NR raw stages, 1 KB of alignment room
static size_t cn_smem_bytes(int NT, int NR) {
  return (size_t)2 * (4 * kTcM + 2 * NT) * kCnCh * 16 + (size_t)NR * (kTcM + NT) * kRawPitch + kTcAlignPad;
}

// K split of the tensor-core product: one CTA per SM, the slice count minimising waves x stages per
// slice (at least 4 stages per slice), and no slice longer than 8192 complex terms, so the FP32 sum in
// tensor memory stays short (slices are added in an FP32 two-sum pair).
void tc_cn_plan(int M, int N, int K, int* nz_out, int* kslice_out) {
  const int ntiles = (N + 255) / 256;
  const int mtiles = (M + kTcM - 1) / kTcM;
  const int tiles = mtiles * ntiles;
  const int kc = kCnKC;
  const int steps = (K + kc - 1) / kc;
  const int maxz = std::max(1, steps / 4);
  const int minz = (steps + 8192 / kc - 1) / (8192 / kc);
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
  const int kslice = ((steps + best_nz - 1) / best_nz) * kc;
  *kslice_out = kslice;
  *nz_out = std::max(1, (K + kslice - 1) / kslice);
}

// Tensor-core path of gemm_cn<float, float, float> (no Hermitian half, no carry): C = conj(A) B^T, the
// K-slice partials in FP32 (a workspace of the context) reduced in a fixed order.
int gemm_cn_tc(Ctx* c, int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, double2* C,
               int ldc, int* err) {
  const int ntiles = (N + 255) / 256;
  const int nt = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
  const int mtiles = (M + kTcM - 1) / kTcM;
  int nz = 1, kslice = kCnKC;
  tc_cn_plan(M, N, K, &nz, &kslice);
  float2* part = static_cast<float2*>(ws_get(c, "tc_parts32", (size_t)nz * M * N * sizeof(float2)));
  if (!part) return PARO_ERR_CUDA;
  int nr = 5;
  while (nr > 3 && cn_smem_bytes(nt, nr) > kTcSmemMax) --nr;
  if (cn_smem_bytes(nt, nr) > kTcSmemMax) return fail(c, PARO_ERR_ARG, "tensor-core product: N tile too wide");
  static int attr_dev[3] = {-1, -1, -1};
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  const void* kf = nr == 5 ? (const void*)k_gemm_cn_tc<5> : nr == 4 ? (const void*)k_gemm_cn_tc<4>
                                                                    : (const void*)k_gemm_cn_tc<3>;
  if (attr_dev[nr - 3] != dev) {
    PARO_CU(c, cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax));
    attr_dev[nr - 3] = dev;
  }
  const dim3 grid(mtiles, ntiles, nz);
  const size_t sm = cn_smem_bytes(nt, nr);
  if (nr == 5)
    k_gemm_cn_tc<5><<<grid, kTcThreads, sm, c->stream>>>(M, N, K, kslice, nt, A, lda, B, ldb, part, err);
  else if (nr == 4)
    k_gemm_cn_tc<4><<<grid, kTcThreads, sm, c->stream>>>(M, N, K, kslice, nt, A, lda, B, ldb, part, err);
  else
    k_gemm_cn_tc<3><<<grid, kTcThreads, sm, c->stream>>>(M, N, K, kslice, nt, A, lda, B, ldb, part, err);
  PARO_LAUNCH(c, "k_gemm_cn_tc");
  return reduce_parts32(c, M, N, nz, part, C, ldc);
}

int reduce_parts32(Ctx* c, int M, int N, int nz, const float2* part, double2* C, int ldc) {
  k_reduce_parts32<<<(M * N + 255) / 256, 256, 0, c->stream>>>(M, N, nz, part, C, ldc);
  PARO_LAUNCH(c, "k_reduce_parts32");
  return PARO_OK;
}

int wx_presplit(Ctx* c, int M, int K, int NT, int KC, const double2* W, int ldw, bool wt, const double* s,
                float4* Wp) {
  const int mtiles = (M + NT - 1) / NT;
  k_wx_presplit<<<dim3(64, mtiles), 256, 0, c->stream>>>(M, K, NT, KC, W, ldw, wt ? 1 : 0, s, Wp);
  PARO_LAUNCH(c, "k_wx_presplit");
  return PARO_OK;
}

}  // namespace paro
