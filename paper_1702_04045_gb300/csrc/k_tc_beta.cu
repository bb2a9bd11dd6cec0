// Tensor-core products with the Kleinman-Bylander projectors as the fixed operand: the inner solves'
// projections P = beta^H x and the update H x += beta (D o P) (Section 2.2's V_nl term, 3xTF32 as in
// k_tc.cu). The projectors do not change between position updates, so their TF32 hi/lo split is formed
// once, in the exact shared-memory image of every pipeline stage ("beta images", two per k-point: one
// for each product's operand layout), and each stage brings its beta tiles in with one cp.async.bulk.
// Roles inside a CTA replace the block-wide barriers of k_tc.cu's kernels: one thread issues the bulk
// copies, one thread the MMAs, and (projections only) six warps stage and split the orbital operand;
// mbarriers order them (every wait bounded, a kernel that gives up sets the context's error flag, waits
// once more for copies in flight and still releases its tensor memory).
#include <algorithm>

#include "paro_ctx.h"
#include "tc_sm100.cuh"

namespace paro {

static const int kBM = 128;             // TMEM lanes per CTA (rows of the A operand)
static const int kBKC = 8;              // complex K values per stage: 4 chunks of 16 bytes
static const int kBCh = 4;
static const int kTileF4 = kBM * kBCh;  // float4 per 128-row tile (8 KB)
static const uint32_t kBPolls = 1u << 24;
static const size_t kBSmemMax = 220 * 1024;

// ---- beta images ----
// projections: block (mt, st) = [hi | lo] of rows p = 128 mt + r, complex k = 8 st + 2c, 2c + 1 of beta[p][k]
__global__ void k_beta_img_cn(int nproj, int npw, int nstage, const float2* __restrict__ beta,
                              float4* __restrict__ img) {
  const int mt = blockIdx.y;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)nstage * kTileF4;
       i += (size_t)gridDim.x * blockDim.x) {
    const int st = (int)(i / kTileF4), u = (int)(i - (size_t)st * kTileF4);
    const int r = u / kBCh, c = u - r * kBCh;
    const int p = mt * kBM + r, k = st * kBKC + 2 * c;
    const float2 z = make_float2(0.f, 0.f);
    const float2 v0 = p < nproj && k < npw ? beta[(size_t)p * npw + k] : z;
    const float2 v1 = p < nproj && k + 1 < npw ? beta[(size_t)p * npw + k + 1] : z;
    float4 h, l;
    tc_split(v0, v1, h, l);
    const size_t base = ((size_t)mt * nstage + st) * 2 * kTileF4;
    const uint32_t o = tc_off(r, c, kBCh) / 16;
    img[base + o] = h;
    img[base + kTileF4 + o] = l;
  }
}

// update: block (nt, st) = [hi | lo] of rows n = 128 nt + r, projectors k = 8 st + 2c, 2c + 1 of beta[k][n]
__global__ void k_beta_img_wx(int nproj, int npw, int nstage, const float2* __restrict__ beta,
                              float4* __restrict__ img) {
  const int nt = blockIdx.y;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)nstage * kTileF4;
       i += (size_t)gridDim.x * blockDim.x) {
    const int st = (int)(i / kTileF4), u = (int)(i - (size_t)st * kTileF4);
    const int c = u / kBM, r = u - c * kBM;  // consecutive threads: consecutive n (coalesced reads)
    const int n = nt * kBM + r, k = st * kBKC + 2 * c;
    const float2 z = make_float2(0.f, 0.f);
    const float2 v0 = n < npw && k < nproj ? beta[(size_t)k * npw + n] : z;
    const float2 v1 = n < npw && k + 1 < nproj ? beta[(size_t)(k + 1) * npw + n] : z;
    float4 h, l;
    tc_split(v0, v1, h, l);
    const size_t base = ((size_t)nt * nstage + st) * 2 * kTileF4;
    const uint32_t o = tc_off(r, c, kBCh) / 16;
    img[base + o] = h;
    img[base + kTileF4 + o] = l;
  }
}

int beta_images(Ctx* c, int ik) {
  Basis& B = c->bases[ik];
  if (B.d_beta_img_cn && B.d_beta_img_wx) return PARO_OK;
  if (!B.d_beta32 || c->nproj <= 0) return fail(c, PARO_ERR_STATE, "tensor-core projector images: no projectors");
  const int mtiles = (c->nproj + kBM - 1) / kBM, ntiles = (B.npw + kBM - 1) / kBM;
  B.img_cn_nstage = (B.npw + kBKC - 1) / kBKC;
  B.img_wx_nstage = (c->nproj + kBKC - 1) / kBKC;
  const size_t ncn = (size_t)mtiles * B.img_cn_nstage * 2 * kTileF4;
  const size_t nwx = (size_t)ntiles * B.img_wx_nstage * 2 * kTileF4;
  PARO_CU(c, cudaMalloc(&B.d_beta_img_cn, ncn * sizeof(float4)));
  PARO_CU(c, cudaMalloc(&B.d_beta_img_wx, nwx * sizeof(float4)));
  k_beta_img_cn<<<dim3(304, mtiles), 256, 0, c->stream>>>(c->nproj, B.npw, B.img_cn_nstage, B.d_beta32,
                                                          B.d_beta_img_cn);
  PARO_LAUNCH(c, "k_beta_img_cn");
  k_beta_img_wx<<<dim3(8, ntiles), 256, 0, c->stream>>>(c->nproj, B.npw, B.img_wx_nstage, B.d_beta32,
                                                        B.d_beta_img_wx);
  PARO_LAUNCH(c, "k_beta_img_wx");
  return PARO_OK;
}

// ---- projections: part[z][m][n] = sum over K slice z of conj(beta[m][k]) x[n][k] ----
// Thread 0 copies the stage's two beta tiles; thread 32 issues the MMAs; warps 2..7 copy x into a raw ring
// NR stages deep (8-byte asynchronous copies: rows of odd length are not 16-byte aligned) and split it into
// four B tiles, B' = x and B'' = (im, -re) (Re conj(a) b = a'.b', Im conj(a) b = a'.b''). Per operand buffer
// b: fullA[b] (the bulk copy's bytes), fullB[b] (192 arrivals), freeb[b] (the MMAs' commit).
static const int kCnbWorkers = 192;
static const int kCnbRawPitch = 80;

template <int NR>
__global__ void __launch_bounds__(256, 1) k_gemm_cn_tcb(int M, int N, int K, int kslice, int NT, int nstage_all,
                                                        const float4* __restrict__ Aimg,
                                                        const float2* __restrict__ X, int ldx,
                                                        float2* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = tc_align1024(smem_dyn);
  const int A_BYTES = 2 * kTileF4 * 16;
  const int BT = NT * kBCh * 16;
  const int BUF = A_BYTES + 4 * BT;
  const int RAW = NT * kCnbRawPitch;
  unsigned char* raw0 = smem + 2 * BUF;
  __shared__ uint64_t fullA[2], fullB[2], freeb[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_wfail[2], s_last_commit, s_last_a[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, m0 = mt * kBM, n0 = blockIdx.y * NT;
  const int k0 = blockIdx.z * kslice, k1 = min(K, k0 + kslice);
  const int nst = k1 > k0 ? (k1 - k0 + kBKC - 1) / kBKC : 0;
  const int gs0 = k0 / kBKC;  // kslice is a multiple of kBKC
  const uint32_t ncols = NT <= 128 ? 256u : 512u;  // Re and Im accumulators, NT columns each
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&fullA[b], 1);
      tc::mbar_init(&fullB[b], kCnbWorkers);
      tc::mbar_init(&freeb[b], 1);
      s_wfail[b] = 0;
      s_last_a[b] = -1;
    }
    s_fail = 0;
    s_last_commit = -1;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t dR = tmem_base, dI = tmem_base + ncols / 2;
  volatile int* vfail = &s_fail;
  if (tid == 0) {  // beta tiles, one bulk copy per stage
    for (int s = 0; s < nst && !*vfail; ++s) {
      const int b = s & 1;
      if (s >= 2 && !tc::mbar_wait(&freeb[b], ((s - 2) >> 1) & 1, kBPolls)) {
        *vfail = 1;
        break;
      }
      tc::mbar_arrive_expect_tx(&fullA[b], (uint32_t)A_BYTES);
      tc::bulk_g2s(smem + b * BUF, Aimg + ((size_t)mt * nstage_all + gs0 + s) * 2 * kTileF4, (uint32_t)A_BYTES,
                   &fullA[b]);
      s_last_a[b] = s;
    }
  } else if (tid == 32) {  // the MMAs
    const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)NT);
    for (int s = 0; s < nst; ++s) {
      const int b = s & 1;
      const uint32_t ph = (uint32_t)(s >> 1) & 1u;
      if (*vfail || !tc::mbar_wait(&fullA[b], ph, kBPolls) || !tc::mbar_wait(&fullB[b], ph, kBPolls)) {
        *vfail = 1;
        break;
      }
      tc::tc_fence_after();
      const uint32_t aH = tc::smem_addr(smem + b * BUF), aL = aH + (uint32_t)A_BYTES / 2, bb = aH + (uint32_t)A_BYTES;
      const uint32_t rH = bb, rL = bb + BT, iH = bb + 2 * BT, iL = bb + 3 * BT;
#pragma unroll
      for (int s2 = 0; s2 < kBCh / 2; ++s2) {
        const uint64_t dAh = tc_desc(aH, s2, kBCh), dAl = tc_desc(aL, s2, kBCh);
        const uint64_t dRh = tc_desc(rH, s2, kBCh), dRl = tc_desc(rL, s2, kBCh);
        const uint64_t dIh = tc_desc(iH, s2, kBCh), dIl = tc_desc(iL, s2, kBCh);
        const uint32_t acc = (s > 0 || s2 > 0) ? 1u : 0u;
        tc::mma_tf32(dR, dAh, dRh, idesc, acc);
        tc::mma_tf32(dR, dAh, dRl, idesc, 1u);
        tc::mma_tf32(dR, dAl, dRh, idesc, 1u);
        tc::mma_tf32(dI, dAh, dIh, idesc, acc);
        tc::mma_tf32(dI, dAh, dIl, idesc, 1u);
        tc::mma_tf32(dI, dAl, dIh, idesc, 1u);
      }
      tc::mma_commit(&freeb[b]);
      s_last_commit = s;
    }
  } else if (warp >= 2) {  // x: raw ring, split into the B tiles
    const int w = tid - 64;
    auto issue = [&](int st) {
      unsigned char* raw = raw0 + (st % NR) * RAW;
      const int kk = k0 + st * kBKC;
      for (int i = w; i < NT * kBKC; i += kCnbWorkers) {
        const int r = i >> 3, kx = i & 7, gk = kk + kx;
        const bool in = n0 + r < N && gk < k1;
        cp_async8(raw + r * kCnbRawPitch + kx * 8, in ? X + (size_t)(n0 + r) * ldx + gk : X, in ? 8 : 0);
      }
    };
#pragma unroll
    for (int p = 0; p < NR - 1; ++p) {
      if (p < nst) issue(p);
      cp_async_commit();
    }
    for (int s = 0; s < nst; ++s) {
      cp_async_wait<NR - 2>();  // this thread's copies of raw stage s have landed
      const int b = s & 1;
      // one worker waits for the buffer; its verdict (and the other roles' failures) reaches every worker
      // through the barrier in a slot of its own, so that all of them leave the loop together
      if (w == 0) {
        int bad = *vfail;
        if (!bad && s >= 2 && !tc::mbar_wait(&freeb[b], ((s - 2) >> 1) & 1, kBPolls)) bad = 1;
        s_wfail[s & 1] = bad;
      }
      tc::named_bar(1, kCnbWorkers);  // raw stage s visible; every worker is past its split of stage s - 1
      if (s_wfail[s & 1]) {
        if (w == 0) *vfail = 1;
        break;
      }
      if (s + NR - 1 < nst) issue(s + NR - 1);  // into the raw slot split at stage s - 1
      cp_async_commit();
      const unsigned char* raw = raw0 + (s % NR) * RAW;
      unsigned char* sB = smem + b * BUF + A_BYTES;
      // unit u -> (row, chunk): 8 consecutive threads take the 8 rows of one core matrix at one chunk
      for (int u = w; u < NT * kBCh; u += kCnbWorkers) {
        const int r = (u & 7) + 8 * (u / (8 * kBCh)), cc = (u >> 3) % kBCh;
        const float4 v = *reinterpret_cast<const float4*>(raw + r * kCnbRawPitch + cc * 16);
        float4 h, l;
        tc_split(make_float2(v.x, v.y), make_float2(v.z, v.w), h, l);
        const uint32_t o = tc_off(r, cc, kBCh);
        *reinterpret_cast<float4*>(sB + o) = h;
        *reinterpret_cast<float4*>(sB + BT + o) = l;
        *reinterpret_cast<float4*>(sB + 2 * BT + o) = make_float4(h.y, -h.x, h.w, -h.z);
        *reinterpret_cast<float4*>(sB + 3 * BT + o) = make_float4(l.y, -l.x, l.w, -l.z);
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&fullB[b]);
    }
    cp_async_wait<0>();  // no copy into shared memory outlives the CTA
  }
  __syncthreads();
  // the last commit covers every MMA issued; copies of beta tiles that no MMA consumed land before exit
  int ok = !*vfail;
  const int lc = s_last_commit;
  if (lc >= 0 && !tc::mbar_wait(&freeb[lc & 1], (uint32_t)(lc >> 1) & 1u, kBPolls)) ok = 0;
  if (lc != nst - 1) ok = 0;
  if (tid == 0)
    for (int b = 0; b < 2; ++b)
      if (s_last_a[b] > lc) tc::mbar_wait(&fullA[b], (uint32_t)(s_last_a[b] >> 1) & 1u, kBPolls);
  ok = __syncthreads_and(ok);
  tc::tc_fence_after();
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
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, ncols);
  }
  if (!ok && tid == 0 && nst > 0) atomicExch(err, 1);
}

// ---- update: Y[m][n] = beta Y[m][n] + sum_k s_k W(k, m) beta_proj[k][n] ----
// D[n][m] = sum_k A[n][k] B[m][k] with A = the beta image of the update (rows n of the N-tile) and B = the
// presplit W tiles of k_wx_presplit (Re D = A'.(Wr, -Wi)', Im D = A'.(Wi, Wr)'). No thread stages an
// operand: thread 0 brings each stage's A and B tiles in with two bulk copies into a ring of NS buffers and
// thread 32 issues the MMAs. Warps 4..7 meanwhile prefetch the CTA's part of Y into L2, so that the
// epilogue's beta Y + D (added in FP32 on the CUDA cores: the tensor core's own accumulation would round
// the small projector term against the large Y) reads it from L2. Every N-tile starts its stage sequence
// at its own offset, so the CTAs do not all read the same B tiles from L2 at once.
__global__ void __launch_bounds__(256, 1) k_gemm_wx_tcb(int M, int N, int NT, int nstage, int NS,
                                                        const float4* __restrict__ Aimg,
                                                        const float4* __restrict__ Wp, float2* __restrict__ Y,
                                                        int ldy, float beta, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = tc_align1024(smem_dyn);
  const int A_BYTES = 2 * kTileF4 * 16;
  const int BT = NT * kBCh * 16;
  const int BUF = A_BYTES + 4 * BT;
  __shared__ uint64_t full[4], freeb[4];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_last_commit, s_last_copy[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = blockIdx.x, mt = blockIdx.y, n0 = nt * kBM, m0 = mt * NT;
  const int rot = nstage > 0 ? nt % nstage : 0;
  const uint32_t ncols = NT <= 128 ? 256u : 512u;
  if (tid == 0) {
    for (int b = 0; b < NS; ++b) {
      tc::mbar_init(&full[b], 1);
      tc::mbar_init(&freeb[b], 1);
      s_last_copy[b] = -1;
    }
    s_fail = 0;
    s_last_commit = -1;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t dR = tmem_base, dI = tmem_base + ncols / 2;
  volatile int* vfail = &s_fail;
  if (tid == 0) {
    for (int s = 0; s < nstage && !*vfail; ++s) {
      const int b = s % NS, st = (s + rot) % nstage;
      if (s >= NS && !tc::mbar_wait(&freeb[b], (uint32_t)(s / NS - 1) & 1u, kBPolls)) {
        *vfail = 1;
        break;
      }
      tc::mbar_arrive_expect_tx(&full[b], (uint32_t)BUF);
      tc::bulk_g2s(smem + b * BUF, Aimg + ((size_t)nt * nstage + st) * 2 * kTileF4, (uint32_t)A_BYTES, &full[b]);
      tc::bulk_g2s(smem + b * BUF + A_BYTES, Wp + ((size_t)mt * nstage + st) * 4 * (size_t)NT * kBCh,
                   (uint32_t)(4 * BT), &full[b]);
      s_last_copy[b] = s;
    }
  } else if (tid == 32) {
    const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)NT);
    for (int s = 0; s < nstage; ++s) {
      const int b = s % NS;
      if (*vfail || !tc::mbar_wait(&full[b], (uint32_t)(s / NS) & 1u, kBPolls)) {
        *vfail = 1;
        break;
      }
      tc::tc_fence_after();
      const uint32_t aH = tc::smem_addr(smem + b * BUF), aL = aH + (uint32_t)A_BYTES / 2, bb = aH + (uint32_t)A_BYTES;
      const uint32_t rH = bb, rL = bb + BT, iH = bb + 2 * BT, iL = bb + 3 * BT;
#pragma unroll
      for (int s2 = 0; s2 < kBCh / 2; ++s2) {
        const uint64_t dAh = tc_desc(aH, s2, kBCh), dAl = tc_desc(aL, s2, kBCh);
        const uint64_t dRh = tc_desc(rH, s2, kBCh), dRl = tc_desc(rL, s2, kBCh);
        const uint64_t dIh = tc_desc(iH, s2, kBCh), dIl = tc_desc(iL, s2, kBCh);
        const uint32_t acc = (s > 0 || s2 > 0) ? 1u : 0u;
        tc::mma_tf32(dR, dAh, dRh, idesc, acc);
        tc::mma_tf32(dR, dAh, dRl, idesc, 1u);
        tc::mma_tf32(dR, dAl, dRh, idesc, 1u);
        tc::mma_tf32(dI, dAh, dIh, idesc, acc);
        tc::mma_tf32(dI, dAh, dIl, idesc, 1u);
        tc::mma_tf32(dI, dAl, dIh, idesc, 1u);
      }
      tc::mma_commit(&freeb[b]);
      s_last_commit = s;
    }
  } else if (warp >= 4 && beta != 0.f) {  // Y's rows n0.. of columns m0.. into L2: one line per 128 bytes
    const int lines = (min(N - n0, kBM) * 8 + 127) / 128;
    for (int i = tid - 128; i < NT * lines; i += 128) {
      const int mm = i / lines, li = i - mm * lines;
      if (m0 + mm < M)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(Y + (size_t)(m0 + mm) * ldy + n0) +
                                                    li * 128));
    }
  }
  __syncthreads();
  int ok = !*vfail;
  const int lc = s_last_commit;
  if (lc >= 0 && !tc::mbar_wait(&freeb[lc % NS], (uint32_t)(lc / NS) & 1u, kBPolls)) ok = 0;
  if (lc != nstage - 1) ok = 0;
  if (tid == 0)
    for (int b = 0; b < NS; ++b)
      if (s_last_copy[b] > lc) tc::mbar_wait(&full[b], (uint32_t)(s_last_copy[b] / NS) & 1u, kBPolls);
  ok = __syncthreads_and(ok);
  tc::tc_fence_after();
  // warps w and w + 4 read TMEM lanes 32 (w % 4) .., columns split between them
  const int lq = warp & 3, half = warp >> 2;
  const int gn = n0 + 32 * lq + lane;
  const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
  for (int cb = 8 * half; cb < NT; cb += 16) {
    float re[8], im[8];
    tc::tmem_ld_x8(dR + lane_off + (uint32_t)cb, re);
    tc::tmem_ld_x8(dI + lane_off + (uint32_t)cb, im);
    if (gn < N && ok) {
      float2 o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {  // all eight loads in flight before the first use
        const int m = m0 + cb + j;
        o[j] = beta != 0.f && m < M ? Y[(size_t)m * ldy + gn] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int m = m0 + cb + j;
        if (m < M) Y[(size_t)m * ldy + gn] = make_float2(beta * o[j].x + re[j], beta * o[j].y + im[j]);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, ncols);
  }
  if (!ok && tid == 0 && nstage > 0) atomicExch(err, 1);
}

// ---- host side ----
static int set_smem_max(Ctx* c, const void* k, int* done_dev) {
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (*done_dev != dev) {
    PARO_CU(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmemMax));
    *done_dev = dev;
  }
  return PARO_OK;
}

static size_t cnb_smem(int NT, int NR) {
  return (size_t)2 * (2 * kTileF4 * 16 + 4 * NT * kBCh * 16) + (size_t)NR * NT * kCnbRawPitch + 1024;
}

int gemm_cn_tc_beta(Ctx* c, int ik, int nb, const float2* x, double2* P, int* err) {
  const Basis& B = c->bases[ik];
  const int M = c->nproj, N = nb, K = B.npw;
  const int ntiles = (N + 255) / 256;
  const int NT = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
  const int mtiles = (M + kBM - 1) / kBM;
  int nz = 1, kslice = kBKC;
  tc_cn_plan(M, N, K, &nz, &kslice);
  float2* part = static_cast<float2*>(ws_get(c, "tc_parts32", (size_t)nz * M * N * sizeof(float2)));
  if (!part) return PARO_ERR_CUDA;
  int nr = 4;
  while (nr > 2 && cnb_smem(NT, nr) > kBSmemMax) --nr;
  if (cnb_smem(NT, nr) > kBSmemMax) return fail(c, PARO_ERR_ARG, "tensor-core projections: N tile too wide");
  static int done[3] = {-1, -1, -1};
  const void* kf = nr == 4 ? (const void*)k_gemm_cn_tcb<4> : nr == 3 ? (const void*)k_gemm_cn_tcb<3>
                                                                     : (const void*)k_gemm_cn_tcb<2>;
  int st;
  if ((st = set_smem_max(c, kf, &done[nr - 2]))) return st;
  const dim3 grid(mtiles, ntiles, nz);
  const size_t sm = cnb_smem(NT, nr);
  if (nr == 4)
    k_gemm_cn_tcb<4><<<grid, 256, sm, c->stream>>>(M, N, K, kslice, NT, B.img_cn_nstage, B.d_beta_img_cn, x, K, part,
                                                   err);
  else if (nr == 3)
    k_gemm_cn_tcb<3><<<grid, 256, sm, c->stream>>>(M, N, K, kslice, NT, B.img_cn_nstage, B.d_beta_img_cn, x, K, part,
                                                   err);
  else
    k_gemm_cn_tcb<2><<<grid, 256, sm, c->stream>>>(M, N, K, kslice, NT, B.img_cn_nstage, B.d_beta_img_cn, x, K, part,
                                                   err);
  PARO_LAUNCH(c, "k_gemm_cn_tcb");
  return reduce_parts32(c, M, N, nz, part, P, N);
}

int gemm_wx_tc_beta(Ctx* c, int ik, int nb, const double2* P, const double* dvec, float2* y, int* err) {
  const Basis& B = c->bases[ik];
  const int M = nb, N = B.npw, K = c->nproj;
  const int mtiles = (M + 255) / 256;
  const int NT = ((M + mtiles - 1) / mtiles + 15) / 16 * 16;
  const int nstage = B.img_wx_nstage;  // (K + 7) / 8
  const size_t tile4 = (size_t)NT * kBCh;
  float4* Wp = static_cast<float4*>(ws_get(c, "tc_wxb_split", (size_t)mtiles * nstage * 4 * tile4 * sizeof(float4)));
  if (!Wp) return PARO_ERR_CUDA;
  const size_t buf = (size_t)2 * kTileF4 * 16 + (size_t)4 * NT * kBCh * 16;
  int ns = 4;
  while (ns > 2 && ns * buf + 1024 > kBSmemMax) --ns;
  if (ns * buf + 1024 > kBSmemMax) return fail(c, PARO_ERR_ARG, "tensor-core update: M tile too wide");
  static int done = -1;
  int st;
  if ((st = set_smem_max(c, (const void*)k_gemm_wx_tcb, &done))) return st;
  if (K > 0 && (st = wx_presplit(c, M, K, NT, kBKC, P, M, false, dvec, Wp))) return st;
  k_gemm_wx_tcb<<<dim3((N + kBM - 1) / kBM, mtiles), 256, ns * buf + 1024, c->stream>>>(
      M, N, NT, nstage, ns, B.d_beta_img_wx, Wp, y, N, 1.0f, err);
  PARO_LAUNCH(c, "k_gemm_wx_tcb");
  return PARO_OK;
}

}  // namespace paro
