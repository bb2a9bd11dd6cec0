// Device helpers shared by the libparo kernels: complex arithmetic on float2/double2 and a batched
// mixed-radix (2, 3, 4, 8) Stockham FFT over lines held in shared memory.
//
// The FFT follows the autosort (Stockham) formulation: stage s with radix R and span Ns reads the R
// inputs j + r N/R of butterfly j, multiplies them by the twiddles W_N^{r k N/(Ns R)} (k = j mod Ns),
// does an R-point DFT in registers and writes the outputs to (j/Ns) Ns R + k + r Ns. Every thread
// keeps its butterflies in registers across a __syncthreads(), so a stage runs in place in one
// shared buffer; the host checks that a stage's butterflies fit the per-thread register budget.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace paro {

template <typename T> struct cx;
template <> struct cx<float> { using t = float2; };
template <> struct cx<double> { using t = double2; };
template <typename T> using cplx = typename cx<T>::t;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) { cplx<T> z; z.x = re; z.y = im; return z; }
template <typename Z> __host__ __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z cconj(Z a) { a.y = -a.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z cmul(Z a, Z b) {
  Z r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename Z, typename S> __host__ __device__ __forceinline__ Z cscale(Z a, S s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename Z> __device__ __forceinline__ Z rot90(Z a) {
  Z r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// Radix plan of one FFT length: n = prod rad[0..nst).
struct FftPlan {
  int n;
  int nst;
  int rad[8];
};

// ---------------------------------------------------------------------------------------------
// R-point DFTs in registers, sign -1 (forward) or +1 (inverse).
// ---------------------------------------------------------------------------------------------
template <typename T, bool INV> __device__ __forceinline__ void dft2(cplx<T>* v) {
  cplx<T> a = v[0], b = v[1];
  v[0] = cadd(a, b); v[1] = csub(a, b);
}

template <typename T, bool INV> __device__ __forceinline__ void dft3(cplx<T>* v) {
  const T s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
  cplx<T> a = cadd(v[1], v[2]);
  cplx<T> d = csub(v[1], v[2]);
  cplx<T> m = csub(v[0], cscale(a, (T)0.5));
  cplx<T> jd = cscale(rot90<INV>(d), s3);
  v[0] = cadd(v[0], a);
  v[1] = cadd(m, jd);
  v[2] = csub(m, jd);
}

template <typename T, bool INV> __device__ __forceinline__ void dft4(cplx<T>* v) {
  cplx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  cplx<T> c = cadd(v[1], v[3]), d = rot90<INV>(csub(v[1], v[3]));
  v[0] = cadd(a, c); v[2] = csub(a, c);
  v[1] = cadd(b, d); v[3] = csub(b, d);
}

template <typename T, bool INV> __device__ __forceinline__ void dft8(cplx<T>* v) {
  const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
  cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, INV>(e);
  dft4<T, INV>(o);
  // o[k] *= exp(-+ 2 pi i k / 8)
  cplx<T> t1 = rot90<INV>(o[1]);                       // -+i o1
  o[1] = cscale(cadd(o[1], t1), h);                    // (1 -+ i)/sqrt2 o1
  o[2] = rot90<INV>(o[2]);                             // -+i o2
  cplx<T> t3 = rot90<INV>(o[3]);
  o[3] = cscale(csub(t3, o[3]), h);                    // (-1 -+ i)/sqrt2 o3
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dft_r(cplx<T>* v) {
  if (R == 2) dft2<T, INV>(v);
  else if (R == 3) dft3<T, INV>(v);
  else if (R == 4) dft4<T, INV>(v);
  else dft8<T, INV>(v);
}

// Butterflies a thread holds per stage: at most 8 complex values in registers.
template <int R> struct MaxUnits { static constexpr int v = R == 2 ? 4 : (R == 8 ? 1 : 2); };

// Line geometry: line l starts at base(l), element j at base(l) + j*es.
struct LinesDirect {  // base = l * ls
  int ls;
  __device__ __forceinline__ int operator()(int l) const { return l * ls; }
};
struct LinesMapped {  // base = map[l] * ls
  const int* map;
  int ls;
  __device__ __forceinline__ int operator()(int l) const { return map[l] * ls; }
};

struct LinesPlanes {  // lines of several planes: base = (l / nper) * pstride + (map ? map[l % nper] : l % nper) * ls
  const int* map;
  int nper, ls, pstride;
  __device__ __forceinline__ int operator()(int l) const {
    const int p = l / nper, r = l - p * nper;
    return p * pstride + (map ? map[r] : r) * ls;
  }
};

// One Stockham stage over lines l0 .. l0+nlines-1 of length n in shared memory s; the caller keeps
// nlines * n/R <= MaxUnits<R> * blockDim.x. LFAST: consecutive threads take consecutive lines (for
// strided lines), else consecutive butterflies of one line.
template <typename T, int R, bool INV, bool LFAST, class LB>
__device__ __forceinline__ void fft_stage(cplx<T>* s, int n, int Ns, int l0, int nlines, int es, LB lb,
                                          const cplx<T>* tw) {
  constexpr int MU = MaxUnits<R>::v;
  const int nbf = n / R;
  const int U = nlines * nbf;
  const int stride = n / (Ns * R);
  cplx<T> v[MU][R];
  int dst[MU];
#pragma unroll
  for (int c = 0; c < MU; ++c) {
    const int u = threadIdx.x + c * blockDim.x;
    dst[c] = -1;
    if (u < U) {
      int l, j;
      if (LFAST) { l = u % nlines; j = u / nlines; } else { l = u / nbf; j = u - l * nbf; }
      const int k = j % Ns;
      const int base = lb(l0 + l);
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = s[base + (j + r * nbf) * es];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cplx<T> w = tw[r * k * stride];
          if (INV) w = cconj(w);
          v[c][r] = cmul(v[c][r], w);
        }
      }
      dft_r<T, R, INV>(v[c]);
      dst[c] = base + ((j / Ns) * Ns * R + k) * es;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < MU; ++c) {
    if (dst[c] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[dst[c] + r * Ns * es] = v[c][r];
    }
  }
  __syncthreads();
}

// One stage over all lines, in groups small enough for the per-thread register budget (the lines of
// different groups are disjoint, so a group may be written before the next one is read).
template <typename T, int R, bool INV, bool LFAST, class LB>
__device__ __forceinline__ void fft_stage_all(cplx<T>* s, int n, int Ns, int nlines, int es, LB lb,
                                              const cplx<T>* tw) {
  int gsz = (MaxUnits<R>::v * (int)blockDim.x) / (n / R);
  if (gsz < 1) gsz = 1;
  for (int l0 = 0; l0 < nlines; l0 += gsz)
    fft_stage<T, R, INV, LFAST>(s, n, Ns, l0, min(gsz, nlines - l0), es, lb, tw);
}

// Full FFT of `nlines` lines (all stages of plan p). tw: twiddles exp(-2 pi i j / n), j < n.
// Requires n/R <= MaxUnits<R> * blockDim.x for every radix R of the plan.
template <typename T, bool INV, bool LFAST, class LB>
__device__ __forceinline__ void fft_lines(cplx<T>* s, const FftPlan& p, int nlines, int es, LB lb, const cplx<T>* tw) {
  int Ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.rad[st];
    if (R == 8) fft_stage_all<T, 8, INV, LFAST>(s, p.n, Ns, nlines, es, lb, tw);
    else if (R == 4) fft_stage_all<T, 4, INV, LFAST>(s, p.n, Ns, nlines, es, lb, tw);
    else if (R == 3) fft_stage_all<T, 3, INV, LFAST>(s, p.n, Ns, nlines, es, lb, tw);
    else fft_stage_all<T, 2, INV, LFAST>(s, p.n, Ns, nlines, es, lb, tw);
    Ns *= R;
  }
}

// Grid-wide barrier for kernels started with cudaLaunchCooperativeKernel (all CTAs co-resident).
// bar[0] counts arrivals, bar[1] is the generation. The wait is bounded: after ~2^24 polls (about a
// second) the CTA sets *err and the barrier returns false, so a kernel can leave instead of hanging.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x * gridDim.y * gridDim.z - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned polls = 0;
      while (*gen == g) {
        if (++polls > (1u << 24) || *(volatile int*)err) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, <= 1024).
// Sum over the CTA in FP32 (valid in thread 0); red: 32 floats of shared memory.
__device__ __forceinline__ float block_sumf(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.f;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// Ampere-style asynchronous copies global -> shared of 8 or 16 bytes; src_bytes = 0 fills the destination
// with zeros (the source is then not read, but must still be a valid address)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// hi + lo += x with the rounding error of hi + x kept exactly (two-sum: six FP32 operations, no branch)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (x - bp);
  hi = s;
}

}  // namespace paro
