// Batched preconditioned CG for the independent source problems of Algorithm 1 step 3 (and the
// correction equations of Algorithm 2 step 3): one system (H - sigma) x_b = rhs_b per orbital b, all
// orbitals advanced together, each with its own step lengths and its own stopping test. Dot products
// are formed per (orbital, chunk) in FP64 and summed in a fixed order by per-orbital kernels, so the
// result does not depend on scheduling.
#include "paro_ctx.h"

namespace paro {

static const int kChunk = 2048;  // plane waves per CTA in the vector kernels
static const int kVT = 256;

// Per-thread sum of the dot-product terms: FP64 for FP64 vectors; for FP32 vectors the FP32 terms are
// added into an FP32 two-sum pair (no FP64 instructions per element, which GB300 issues at 1/64 rate,
// and no accumulation error beyond the terms' own FP32 rounding).
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) { two_sum_acc(hi, lo, v); }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// r = b - Ax (or b when ax == nullptr), z = M r, p = z; partials of <r,z> and |r|^2
template <typename T>
__global__ void __launch_bounds__(kVT) k_pcg_init(int npw, int nchunk, const cplx<T>* __restrict__ bvec,
                                                  const cplx<T>* __restrict__ ax, cplx<T>* __restrict__ r,
                                                  cplx<T>* __restrict__ p, const T* __restrict__ kin, T pshift,
                                                  double* __restrict__ prz, double* __restrict__ prr) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  const size_t o = (size_t)b * npw;
  DotAcc<T> az, ar;
  const int g0 = ch * kChunk, g1 = min(npw, g0 + kChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kVT) {
    cplx<T> rv = bvec[o + g];
    if (ax) rv = csub(rv, ax[o + g]);
    const T m = (T)1 / (kin[g] + pshift);
    r[o + g] = rv;
    p[o + g] = cscale(rv, m);
    const T q = rv.x * rv.x + rv.y * rv.y;
    ar.add(q);
    az.add(q * m);
  }
  double rz = block_sum(az.value(), red);
  if (threadIdx.x == 0) prz[(size_t)b * nchunk + ch] = rz;
  double rr = block_sum(ar.value(), red);
  if (threadIdx.x == 0) prr[(size_t)b * nchunk + ch] = rr;
}

// The start of the source solves from x0 = psi with H psi known: rhs = f psi, r = rhs - (H psi - sigma psi),
// z = M r, p = z, partials of <r,z> and |r|^2, and x = psi, hx = H psi (hx may be null) in the same pass
template <typename T>
__global__ void __launch_bounds__(kVT) k_pcg_init_src(int npw, int nchunk, const cplx<T>* __restrict__ psi,
                                                      const cplx<T>* __restrict__ hpsi, const double* __restrict__ f,
                                                      T sigma, cplx<T>* __restrict__ x, cplx<T>* __restrict__ hx,
                                                      cplx<T>* __restrict__ r, cplx<T>* __restrict__ p,
                                                      const T* __restrict__ kin, T pshift, double* __restrict__ prz,
                                                      double* __restrict__ prr) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  const size_t o = (size_t)b * npw;
  const T fb = (T)f[b];
  DotAcc<T> az, ar;
  const int g0 = ch * kChunk, g1 = min(npw, g0 + kChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kVT) {
    const cplx<T> v = psi[o + g], h = hpsi[o + g];
    const cplx<T> ap = mk<T>(h.x - sigma * v.x, h.y - sigma * v.y);
    const cplx<T> rv = csub(cscale(v, fb), ap);
    const T m = (T)1 / (kin[g] + pshift);
    x[o + g] = v;
    if (hx) hx[o + g] = h;
    r[o + g] = rv;
    p[o + g] = cscale(rv, m);
    const T q = rv.x * rv.x + rv.y * rv.y;
    ar.add(q);
    az.add(q * m);
  }
  double rz = block_sum(az.value(), red);
  if (threadIdx.x == 0) prz[(size_t)b * nchunk + ch] = rz;
  double rr = block_sum(ar.value(), red);
  if (threadIdx.x == 0) prr[(size_t)b * nchunk + ch] = rr;
}

__global__ void k_pcg_band_init(int nb, int nchunk, const double* __restrict__ prz, const double* __restrict__ prr,
                                double* __restrict__ rz, double* __restrict__ r0n, int* __restrict__ active,
                                int* __restrict__ its, int* __restrict__ nactive) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double a = 0.0, q = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) {
    a += prz[(size_t)b * nchunk + ch];
    q += prr[(size_t)b * nchunk + ch];
  }
  rz[b] = a;
  r0n[b] = sqrt(q);
  active[b] = q > 0.0 ? 1 : 0;
  its[b] = 0;
  if (q > 0.0) atomicAdd(nactive, 1);
}

// partials of Re <p, Ap>
template <typename T>
__global__ void __launch_bounds__(kVT) k_pcg_dot(int npw, int nchunk, const cplx<T>* __restrict__ p,
                                                 const cplx<T>* __restrict__ ap, const int* __restrict__ active,
                                                 double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (!active[b]) return;
  const size_t o = (size_t)b * npw;
  DotAcc<T> acc;
  const int g0 = ch * kChunk, g1 = min(npw, g0 + kChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kVT) {
    const cplx<T> u = p[o + g], v = ap[o + g];
    acc.add(u.x * v.x + u.y * v.y);
  }
  double s = block_sum(acc.value(), red);
  if (threadIdx.x == 0) part[(size_t)b * nchunk + ch] = s;
}

__global__ void k_pcg_band_alpha(int nb, int nchunk, const double* __restrict__ part, const double* __restrict__ rz,
                                 const int* __restrict__ active, double* __restrict__ alpha, int* __restrict__ bad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (!active[b]) {
    alpha[b] = 0.0;
    return;
  }
  double s = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) s += part[(size_t)b * nchunk + ch];
  if (!(s > 0.0) || !isfinite(s)) {
    atomicExch(bad, b + 1);
    alpha[b] = 0.0;
    return;
  }
  alpha[b] = rz[b] / s;
}

// x += alpha p, r -= alpha Ap; partials of |r|^2 and <r, M r>
template <typename T>
__global__ void __launch_bounds__(kVT) k_pcg_update(int npw, int nchunk, cplx<T>* __restrict__ x,
                                                    cplx<T>* __restrict__ r, const cplx<T>* __restrict__ p,
                                                    const cplx<T>* __restrict__ ap, const T* __restrict__ kin,
                                                    T pshift, const double* __restrict__ alpha,
                                                    const int* __restrict__ active, double* __restrict__ prr,
                                                    double* __restrict__ prz, cplx<T>* __restrict__ hx, T sigma) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (!active[b]) return;
  const T a = (T)alpha[b];
  const size_t o = (size_t)b * npw;
  DotAcc<T> ar, az;
  const int g0 = ch * kChunk, g1 = min(npw, g0 + kChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kVT) {
    const cplx<T> pv = p[o + g], av = ap[o + g];
    cplx<T> xv = x[o + g], rv = r[o + g];
    xv.x += a * pv.x; xv.y += a * pv.y;
    rv.x -= a * av.x; rv.y -= a * av.y;
    x[o + g] = xv;
    r[o + g] = rv;
    if (hx) {  // H x follows x: H p = ap + sigma p
      cplx<T> hv = hx[o + g];
      hv.x += a * (av.x + sigma * pv.x);
      hv.y += a * (av.y + sigma * pv.y);
      hx[o + g] = hv;
    }
    const T q = rv.x * rv.x + rv.y * rv.y;
    ar.add(q);
    az.add(q * ((T)1 / (kin[g] + pshift)));
  }
  double rr = block_sum(ar.value(), red);
  if (threadIdx.x == 0) prr[(size_t)b * nchunk + ch] = rr;
  double rz = block_sum(az.value(), red);
  if (threadIdx.x == 0) prz[(size_t)b * nchunk + ch] = rz;
}

__global__ void k_pcg_band_beta(int nb, int nchunk, const double* __restrict__ prr, const double* __restrict__ prz,
                                const double* __restrict__ r0n, double tol, double* __restrict__ rz,
                                int* __restrict__ active, int* __restrict__ its, double* __restrict__ beta,
                                int* __restrict__ still_out, int* __restrict__ nactive) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (!active[b]) {
    still_out[b] = 0;
    beta[b] = 0.0;
    return;
  }
  double q = 0.0, a = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) {
    q += prr[(size_t)b * nchunk + ch];
    a += prz[(size_t)b * nchunk + ch];
  }
  its[b] += 1;
  const int still = sqrt(q) > tol * r0n[b] ? 1 : 0;
  beta[b] = still ? a / rz[b] : 0.0;
  if (still) rz[b] = a;
  still_out[b] = still;
  if (still) atomicAdd(nactive, 1);
}

// p = M r + beta p for the orbitals still active
template <typename T>
__global__ void __launch_bounds__(kVT) k_pcg_pupdate(int npw, cplx<T>* __restrict__ p, const cplx<T>* __restrict__ r,
                                                     const T* __restrict__ kin, T pshift,
                                                     const double* __restrict__ beta, const int* __restrict__ still) {
  const int b = blockIdx.y, ch = blockIdx.x;
  if (!still[b]) return;
  const T bt = (T)beta[b];
  const size_t o = (size_t)b * npw;
  const int g0 = ch * kChunk, g1 = min(npw, g0 + kChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kVT) {
    const T m = (T)1 / (kin[g] + pshift);
    const cplx<T> rv = r[o + g], pv = p[o + g];
    p[o + g] = mk<T>(m * rv.x + bt * pv.x, m * rv.y + bt * pv.y);
  }
}

// y_b = f_b x_b
template <typename T>
__global__ void k_scale_rows(int npw, const cplx<T>* __restrict__ x, const double* __restrict__ f,
                             cplx<T>* __restrict__ y) {
  const int b = blockIdx.y;
  const T s = (T)f[b];
  const size_t o = (size_t)b * npw;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x)
    y[o + g] = cscale(x[o + g], s);
}

template <typename T>
int scale_rows(Ctx* c, int nb, int npw, const cplx<T>* x, const double* f_dev, cplx<T>* y) {
  k_scale_rows<T><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, x, f_dev, y);
  PARO_LAUNCH(c, "k_scale_rows");
  return PARO_OK;
}

template <typename T> static const T* kin_ptr(const Basis& b);
template <> const double* kin_ptr<double>(const Basis& b) { return b.d_kin; }
template <> const float* kin_ptr<float>(const Basis& b) { return b.d_kin32; }

// ap_b = hx_b - sigma x_b: (H - sigma) x from a known H x
template <typename T>
__global__ void k_shift_known(int npw, const cplx<T>* __restrict__ hx, const cplx<T>* __restrict__ x, T sigma,
                              cplx<T>* __restrict__ ap) {
  const size_t o = (size_t)blockIdx.y * npw;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
    const cplx<T> h = hx[o + g], v = x[o + g];
    ap[o + g] = mk<T>(h.x - sigma * v.x, h.y - sigma * v.y);
  }
}

// Solves (H - sigma_k) x_b = rhs_b for b < nb. On entry x holds the start vectors (ignored when
// x0_zero), on exit the approximate solutions. Every orbital stops once ||r_b|| <= rel_tol ||r_b^0||
// or after max_it steps; iters (host, may be null) receives the steps taken. hx0 (may be null): H x
// of the start vectors when the caller already has it (the orbitals' H psi from the last
// Rayleigh-Ritz step), which saves the first H application. hx (may be null; needs hx0 or x0_zero):
// receives H x of the solutions, carried along the iteration from the products the solver forms anyway.
// x0src, fsrc (both or neither): rhs = diag(fsrc) x0src and x0 = x0src, formed in the first pass (rhs is then
// not read; needs hx0 = H x0src).
template <typename T>
int pcg_run(Ctx* c, int ik, int nb, const cplx<T>* rhs, cplx<T>* x, bool x0_zero, double rel_tol, int max_it,
            int* iters, const cplx<T>* hx0, cplx<T>* hx, const cplx<T>* x0src, const double* fsrc) {
  ProfTag tag(c, "pcg");
  TcScope tcs(c);  // the inner solves tolerate the 3xTF32 products
  const Basis& B = c->bases[ik];
  const int npw = B.npw;
  const int nchunk = (npw + kChunk - 1) / kChunk;
  int st = veff_stats(c);
  if (st) return st;
  const double sigma = c->sigma_k[ik];
  const T pshift = (T)(c->vmean - sigma);
  const size_t vb = (size_t)nb * npw * sizeof(cplx<T>);
  const bool f64 = sizeof(T) == 8;
  cplx<T>* r = static_cast<cplx<T>*>(ws_get(c, f64 ? "pcg_r64" : "pcg_r32", vb));
  cplx<T>* p = static_cast<cplx<T>*>(ws_get(c, f64 ? "pcg_p64" : "pcg_p32", vb));
  cplx<T>* ap = static_cast<cplx<T>*>(ws_get(c, f64 ? "pcg_ap64" : "pcg_ap32", vb));
  double* prz = static_cast<double*>(ws_get(c, "pcg_prz", (size_t)nb * nchunk * sizeof(double)));
  double* prr = static_cast<double*>(ws_get(c, "pcg_prr", (size_t)nb * nchunk * sizeof(double)));
  double* band = static_cast<double*>(ws_get(c, "pcg_band", (size_t)nb * 4 * sizeof(double)));
  int* ib = static_cast<int*>(ws_get(c, "pcg_int", (size_t)(nb * 3 + 4) * sizeof(int)));
  if (!r || !p || !ap || !prz || !prr || !band || !ib) return PARO_ERR_CUDA;
  double *rz = band, *r0n = band + nb, *alpha = band + 2 * nb, *beta = band + 3 * nb;
  int *active = ib, *its = ib + nb, *still = ib + 2 * nb, *flags = ib + 3 * nb;  // flags: nactive, bad
  const dim3 gv(nchunk, nb);
  const int tb = (nb + 127) / 128;
  PARO_CU(c, cudaMemsetAsync(flags, 0, 2 * sizeof(int), c->stream));
  if (fsrc) {
    if (!x0src || !hx0 || x0_zero) return fail(c, PARO_ERR_ARG, "pcg_run: the source form needs x0 and H x0");
    k_pcg_init_src<T><<<gv, kVT, 0, c->stream>>>(npw, nchunk, x0src, hx0, fsrc, (T)sigma, x, hx, r, p, kin_ptr<T>(B),
                                                 pshift, prz, prr);
    PARO_LAUNCH(c, "k_pcg_init_src");
  } else {
    if (hx) {
      if (x0_zero) PARO_CU(c, cudaMemsetAsync(hx, 0, vb, c->stream));
      else if (hx0) PARO_CU(c, cudaMemcpyAsync(hx, hx0, vb, cudaMemcpyDeviceToDevice, c->stream));
      else return fail(c, PARO_ERR_ARG, "pcg_run: H x of the solutions needs H x of the start vectors");
    }
    if (!x0_zero && hx0) {
      k_shift_known<T><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, hx0, x, (T)sigma, ap);
      PARO_LAUNCH(c, "k_shift_known");
    } else if (!x0_zero) {
      st = apply_h<T>(c, ik, nb, x, ap, sigma, nullptr);
      if (st) return st;
    } else {
      PARO_CU(c, cudaMemsetAsync(x, 0, vb, c->stream));
    }
    k_pcg_init<T><<<gv, kVT, 0, c->stream>>>(npw, nchunk, rhs, x0_zero ? nullptr : ap, r, p, kin_ptr<T>(B), pshift,
                                             prz, prr);
    PARO_LAUNCH(c, "k_pcg_init");
  }
  k_pcg_band_init<<<tb, 128, 0, c->stream>>>(nb, nchunk, prz, prr, rz, r0n, active, its, flags);
  PARO_LAUNCH(c, "k_pcg_band_init");
  // the first step runs without reading the active count back: every orbital with a nonzero initial
  // residual is active, and the kernels pass over the others
  int hflags[2] = {1, 0};
  for (int it = 0; it < max_it && hflags[0] > 0; ++it) {
    st = apply_h<T>(c, ik, nb, p, ap, sigma, active);
    if (st) return st;
    cudaEvent_t ev = prof_begin(c);
    k_pcg_dot<T><<<gv, kVT, 0, c->stream>>>(npw, nchunk, p, ap, active, prz);
    PARO_LAUNCH(c, "k_pcg_dot");
    k_pcg_band_alpha<<<tb, 128, 0, c->stream>>>(nb, nchunk, prz, rz, active, alpha, flags + 1);
    PARO_LAUNCH(c, "k_pcg_band_alpha");
    k_pcg_update<T><<<gv, kVT, 0, c->stream>>>(npw, nchunk, x, r, p, ap, kin_ptr<T>(B), pshift, alpha, active, prr,
                                               prz, hx, (T)sigma);
    PARO_LAUNCH(c, "k_pcg_update");
    PARO_CU(c, cudaMemsetAsync(flags, 0, sizeof(int), c->stream));
    k_pcg_band_beta<<<tb, 128, 0, c->stream>>>(nb, nchunk, prr, prz, r0n, rel_tol, rz, active, its, beta, still,
                                               flags);
    PARO_LAUNCH(c, "k_pcg_band_beta");
    k_pcg_pupdate<T><<<gv, kVT, 0, c->stream>>>(npw, p, r, kin_ptr<T>(B), pshift, beta, still);
    PARO_LAUNCH(c, "k_pcg_pupdate");
    prof_end(c, f64 ? "pcg_vector<f64>" : "pcg_vector<f32>", ev);
    PARO_CU(c, cudaMemcpyAsync(active, still, nb * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
    PARO_CU(c, cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PARO_CU(c, cudaStreamSynchronize(c->stream));
    if (hflags[1]) return fail(c, PARO_ERR_BREAKDOWN, "PCG breakdown (p^H A p <= 0 or not finite) in orbital " +
                                                         std::to_string(hflags[1] - 1));
  }
  if (iters) {
    PARO_CU(c, cudaMemcpyAsync(iters, its, nb * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PARO_CU(c, cudaStreamSynchronize(c->stream));
  }
  return PARO_OK;
}

template int pcg_run<double>(Ctx*, int, int, const double2*, double2*, bool, double, int, int*, const double2*,
                             double2*, const double2*, const double*);
template int pcg_run<float>(Ctx*, int, int, const float2*, float2*, bool, double, int, int*, const float2*, float2*,
                            const float2*, const double*);
template int scale_rows<double>(Ctx*, int, int, const double2*, const double*, double2*);
template int scale_rows<float>(Ctx*, int, int, const float2*, const double*, float2*);

}  // namespace paro
