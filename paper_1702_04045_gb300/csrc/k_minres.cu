// Batched preconditioned MINRES for the projected correction equations of Algorithm 3 (MParO II), step 3:
//   (I - P_b)(H - eps_b)(I - P_b) e_b = -(H psi_b - eps_b psi_b),  P_b = |psi_b><psi_b|,
// one Hermitian, generally indefinite system per orbital b on the complement of psi_b, all orbitals
// advanced together with their own Lanczos and Givens scalars and their own stopping test. The
// preconditioner is (I - P_b) D (I - P_b) with D = diag(|k+G|^2/2 + mean V - sigma)^{-1} (the PCG
// preconditioner), positive definite on that complement. Lanczos runs in the M^{-1} inner product and
// the tridiagonal is reduced by Givens rotations (Paige and Saunders); eta_b estimates the preconditioned
// residual norm, and an orbital stops once |eta_b| <= rel_tol |eta_b^0| or after max_it steps. Dot
// products are formed per (orbital, chunk) and summed in a fixed order by per-orbital kernels.
#include <algorithm>

#include "paro_ctx.h"

namespace paro {

static const int kMChunk = 2048;  // plane waves per CTA in the vector kernels
static const int kMT = 256;

template <typename T> struct MAcc;  // per-thread sums: FP64, or an FP32 two-sum pair for FP32 vectors
template <> struct MAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct MAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) { two_sum_acc(hi, lo, v); }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Band scalars (double), nb each: gamma, gamma_old, eta, eta0, c, c_old, s, s_old, delta, a1, a2, a3,
// xcoef; projection coefficients cre, cim.
enum { MG = 0, MGO, META, META0, MC, MCO, MS, MSO, MDEL, MA1, MA2, MA3, MXC, MCRE, MCIM, MNS };

// partials of <psi_b, u_b> = sum conj(psi) u (re, im) over one chunk; part[(b * nchunk + ch) * 2 + {0,1}]
template <typename T>
__device__ __forceinline__ void dot_c_partial(const cplx<T>* psi, const cplx<T>* u, size_t o, int g0, int g1,
                                              double* part, int b, int nchunk, int ch, double* red) {
  MAcc<T> ar, ai;
  for (int g = g0 + threadIdx.x; g < g1; g += kMT) {
    const cplx<T> p = psi[o + g], v = u[o + g];
    ar.add(p.x * v.x + p.y * v.y);
    ai.add(p.x * v.y - p.y * v.x);
  }
  const double sr = block_sum(ar.value(), red);
  if (threadIdx.x == 0) part[((size_t)b * nchunk + ch) * 2] = sr;
  const double si = block_sum(ai.value(), red);
  if (threadIdx.x == 0) part[((size_t)b * nchunk + ch) * 2 + 1] = si;
}

// v = -(hpsi - eps psi); partial <psi, v>
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_rhs(int npw, int nchunk, const cplx<T>* __restrict__ psi,
                                               const cplx<T>* __restrict__ hpsi, const double* __restrict__ eps,
                                               cplx<T>* __restrict__ v, double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  const size_t o = (size_t)b * npw;
  const T e = (T)eps[b];
  const int g0 = ch * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kMT) {
    const cplx<T> p = psi[o + g], h = hpsi[o + g];
    v[o + g] = mk<T>(e * p.x - h.x, e * p.y - h.y);
  }
  __syncthreads();
  dot_c_partial<T>(psi, v, o, g0, g1, part, b, nchunk, ch, red);
}

// per band: c = sum over chunks of the complex partials (fixed order)
__global__ void k_mr_band_c(int nb, int nchunk, const double* __restrict__ part, const int* __restrict__ active,
                            double* __restrict__ sc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || (active && !active[b])) return;
  double re = 0.0, im = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) {
    re += part[((size_t)b * nchunk + ch) * 2];
    im += part[((size_t)b * nchunk + ch) * 2 + 1];
  }
  sc[MCRE * nb + b] = re;
  sc[MCIM * nb + b] = im;
}

// u -= c psi; y = D u; partial <psi, y>   (u: the right-hand side or the new Lanczos vector, in place)
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_proj_prec(int npw, int nchunk, int nb, const cplx<T>* __restrict__ psi,
                                                     cplx<T>* __restrict__ u, int project_u, cplx<T>* __restrict__ y,
                                                     const T* __restrict__ kin, T pshift,
                                                     const double* __restrict__ sc, const int* __restrict__ active,
                                                     double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (active && !active[b]) return;
  const size_t o = (size_t)b * npw;
  const T cr = (T)sc[MCRE * nb + b], ci = (T)sc[MCIM * nb + b];
  const int g0 = ch * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kMT) {
    cplx<T> w = u[o + g];
    if (project_u) {
      const cplx<T> p = psi[o + g];
      w.x -= cr * p.x - ci * p.y;
      w.y -= cr * p.y + ci * p.x;
      u[o + g] = w;
    }
    const T m = (T)1 / (kin[g] + pshift);
    y[o + g] = mk<T>(m * w.x, m * w.y);
  }
  __syncthreads();
  dot_c_partial<T>(psi, y, o, g0, g1, part, b, nchunk, ch, red);
}

// z = y - c psi (in place); partial Re <z, v>
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_zproj(int npw, int nchunk, int nb, const cplx<T>* __restrict__ psi,
                                                 cplx<T>* __restrict__ y, const cplx<T>* __restrict__ v,
                                                 const double* __restrict__ sc, const int* __restrict__ active,
                                                 double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (active && !active[b]) return;
  const size_t o = (size_t)b * npw;
  const T cr = (T)sc[MCRE * nb + b], ci = (T)sc[MCIM * nb + b];
  MAcc<T> acc;
  const int g0 = ch * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kMT) {
    const cplx<T> p = psi[o + g], vv = v[o + g];
    cplx<T> z = y[o + g];
    z.x -= cr * p.x - ci * p.y;
    z.y -= cr * p.y + ci * p.x;
    y[o + g] = z;
    acc.add(z.x * vv.x + z.y * vv.y);
  }
  const double s = block_sum(acc.value(), red);
  if (threadIdx.x == 0) part[(size_t)b * nchunk + ch] = s;
}

// start: gamma = sqrt(<z, v>), eta = eta0 = gamma, Givens state reset; active where gamma > 0
__global__ void k_mr_band_start(int nb, int nchunk, const double* __restrict__ part, double* __restrict__ sc,
                                int* __restrict__ active, int* __restrict__ its, int* __restrict__ nactive) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double q = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) q += part[(size_t)b * nchunk + ch];
  const double g = q > 0.0 && isfinite(q) ? sqrt(q) : 0.0;
  sc[MG * nb + b] = g;
  sc[MGO * nb + b] = 1.0;
  sc[META * nb + b] = g;
  sc[META0 * nb + b] = g;
  sc[MC * nb + b] = 1.0;
  sc[MCO * nb + b] = 1.0;
  sc[MS * nb + b] = 0.0;
  sc[MSO * nb + b] = 0.0;
  active[b] = g > 0.0 ? 1 : 0;
  its[b] = 0;
  if (g > 0.0) atomicAdd(nactive, 1);
}

// zn = z / gamma; x = w = w_old = v_old = 0
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_init_vectors(int npw, int nb, const double* __restrict__ sc,
                                                        cplx<T>* __restrict__ zn, cplx<T>* __restrict__ x,
                                                        cplx<T>* __restrict__ w, cplx<T>* __restrict__ wo,
                                                        cplx<T>* __restrict__ vo) {
  const int b = blockIdx.y;
  const size_t o = (size_t)b * npw;
  const double g = sc[MG * nb + b];
  const T inv = g > 0.0 ? (T)(1.0 / g) : (T)0;
  const int g0 = blockIdx.x * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int gi = g0 + threadIdx.x; gi < g1; gi += kMT) {
    zn[o + gi] = cscale(zn[o + gi], inv);
    x[o + gi] = w[o + gi] = wo[o + gi] = vo[o + gi] = mk<T>(0, 0);
  }
}

// t = H zn - eps zn (in az); partial <psi, t>
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_shift(int npw, int nchunk, const cplx<T>* __restrict__ psi,
                                                 const cplx<T>* __restrict__ zn, cplx<T>* __restrict__ az,
                                                 const double* __restrict__ eps, const int* __restrict__ active,
                                                 double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (!active[b]) return;
  const size_t o = (size_t)b * npw;
  const T e = (T)eps[b];
  const int g0 = ch * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kMT) {
    const cplx<T> h = az[o + g], z = zn[o + g];
    az[o + g] = mk<T>(h.x - e * z.x, h.y - e * z.y);
  }
  __syncthreads();
  dot_c_partial<T>(psi, az, o, g0, g1, part, b, nchunk, ch, red);
}

// az = t - c psi; partial delta = Re <az, zn>
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_delta(int npw, int nchunk, int nb, const cplx<T>* __restrict__ psi,
                                                 const cplx<T>* __restrict__ zn, cplx<T>* __restrict__ az,
                                                 const double* __restrict__ sc, const int* __restrict__ active,
                                                 double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (!active[b]) return;
  const size_t o = (size_t)b * npw;
  const T cr = (T)sc[MCRE * nb + b], ci = (T)sc[MCIM * nb + b];
  MAcc<T> acc;
  const int g0 = ch * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += kMT) {
    const cplx<T> p = psi[o + g], z = zn[o + g];
    cplx<T> t = az[o + g];
    t.x -= cr * p.x - ci * p.y;
    t.y -= cr * p.y + ci * p.x;
    az[o + g] = t;
    acc.add(t.x * z.x + t.y * z.y);
  }
  const double s = block_sum(acc.value(), red);
  if (threadIdx.x == 0) part[(size_t)b * nchunk + ch] = s;
}

__global__ void k_mr_band_delta(int nb, int nchunk, const double* __restrict__ part, const int* __restrict__ active,
                                double* __restrict__ sc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !active[b]) return;
  double d = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) d += part[(size_t)b * nchunk + ch];
  sc[MDEL * nb + b] = d;
}

// v_new = az - (delta/gamma) v - (gamma/gamma_old) v_old, written over v_old; y = D v_new; partial <psi, y>
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_lanczos(int npw, int nchunk, int nb, const cplx<T>* __restrict__ psi,
                                                   const cplx<T>* __restrict__ az, const cplx<T>* __restrict__ v,
                                                   cplx<T>* __restrict__ vo, cplx<T>* __restrict__ y,
                                                   const T* __restrict__ kin, T pshift, const double* __restrict__ sc,
                                                   const int* __restrict__ active, double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (!active[b]) return;
  const size_t o = (size_t)b * npw;
  const double g = sc[MG * nb + b];
  const T a = (T)(sc[MDEL * nb + b] / g), bb = (T)(g / sc[MGO * nb + b]);
  const int g0 = ch * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int gi = g0 + threadIdx.x; gi < g1; gi += kMT) {
    const cplx<T> t = az[o + gi], v1 = v[o + gi], v0 = vo[o + gi];
    const cplx<T> vn = mk<T>(t.x - a * v1.x - bb * v0.x, t.y - a * v1.y - bb * v0.y);
    vo[o + gi] = vn;
    const T m = (T)1 / (kin[gi] + pshift);
    y[o + gi] = mk<T>(m * vn.x, m * vn.y);
  }
  __syncthreads();
  dot_c_partial<T>(psi, y, o, g0, g1, part, b, nchunk, ch, red);
}

// gamma_new, the Givens rotation, eta and the stopping test
__global__ void k_mr_band_givens(int nb, int nchunk, const double* __restrict__ part, double tol,
                                 const int* __restrict__ active, double* __restrict__ sc, int* __restrict__ its,
                                 int* __restrict__ still, int* __restrict__ nactive, int* __restrict__ bad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (!active[b]) {
    still[b] = 0;
    return;
  }
  double q = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) q += part[(size_t)b * nchunk + ch];
  if (!isfinite(q)) {
    atomicExch(bad, b + 1);
    still[b] = 0;
    return;
  }
  const double gn = q > 0.0 ? sqrt(q) : 0.0;
  const double g = sc[MG * nb + b], d = sc[MDEL * nb + b];
  const double c = sc[MC * nb + b], co = sc[MCO * nb + b], s = sc[MS * nb + b], so = sc[MSO * nb + b];
  const double a0 = c * d - co * s * g;
  const double a1 = sqrt(a0 * a0 + gn * gn);
  const double a2 = s * d + co * c * g;
  const double a3 = so * g;
  if (!(a1 > 0.0) || !isfinite(a1)) {
    atomicExch(bad, b + 1);
    still[b] = 0;
    return;
  }
  const double cn = a0 / a1, sn = gn / a1;
  const double eta = sc[META * nb + b];
  sc[MA1 * nb + b] = a1;
  sc[MA2 * nb + b] = a2;
  sc[MA3 * nb + b] = a3;
  sc[MXC * nb + b] = cn * eta;
  sc[MGO * nb + b] = g;
  sc[MG * nb + b] = gn;
  sc[MCO * nb + b] = c;
  sc[MC * nb + b] = cn;
  sc[MSO * nb + b] = s;
  sc[MS * nb + b] = sn;
  const double en = -sn * eta;
  sc[META * nb + b] = en;
  its[b] += 1;
  const int st = fabs(en) > tol * sc[META0 * nb + b] && gn > 0.0 ? 1 : 0;
  still[b] = st;
  if (st) atomicAdd(nactive, 1);
}

// w_new = (zn - a3 w_old - a2 w) / a1 over w_old; x += xcoef w_new; zn = z_new / gamma_new
template <typename T>
__global__ void __launch_bounds__(kMT) k_mr_update(int npw, int nb, cplx<T>* __restrict__ zn,
                                                  const cplx<T>* __restrict__ znew, const cplx<T>* __restrict__ w,
                                                  cplx<T>* __restrict__ wo, cplx<T>* __restrict__ x,
                                                  const double* __restrict__ sc, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const size_t o = (size_t)b * npw;
  const T ia1 = (T)(1.0 / sc[MA1 * nb + b]), a2 = (T)sc[MA2 * nb + b], a3 = (T)sc[MA3 * nb + b];
  const T xc = (T)sc[MXC * nb + b];
  const double gn = sc[MG * nb + b];
  const T ig = gn > 0.0 ? (T)(1.0 / gn) : (T)0;
  const int g0 = blockIdx.x * kMChunk, g1 = min(npw, g0 + kMChunk);
  for (int gi = g0 + threadIdx.x; gi < g1; gi += kMT) {
    const cplx<T> z = zn[o + gi], w1 = w[o + gi], w0 = wo[o + gi];
    const cplx<T> wn = mk<T>((z.x - a3 * w0.x - a2 * w1.x) * ia1, (z.y - a3 * w0.y - a2 * w1.y) * ia1);
    wo[o + gi] = wn;
    cplx<T> xv = x[o + gi];
    xv.x += xc * wn.x;
    xv.y += xc * wn.y;
    x[o + gi] = xv;
    zn[o + gi] = cscale(znew[o + gi], ig);
  }
}

template <typename T> static const T* kin_of_b(const Basis& b);
template <> const double* kin_of_b<double>(const Basis& b) { return b.d_kin; }
template <> const float* kin_of_b<float>(const Basis& b) { return b.d_kin32; }

// The corrections e_b (in e) of Algorithm 3 for the nb orbitals psi of k-point ik with H psi in hpsi and
// the Ritz values eps (host). iters (host, may be null): the steps each orbital took.
template <typename T>
int minres_run(Ctx* c, int ik, int nb, const cplx<T>* psi, const cplx<T>* hpsi, const double* eps, cplx<T>* e,
               double rel_tol, int max_it, int* iters) {
  ProfTag tag(c, "minres");
  TcScope tcs(c);  // inexact inner solves: the 3xTF32 tensor-core products are accurate enough
  const Basis& B = c->bases[ik];
  const int npw = B.npw;
  const int nchunk = (npw + kMChunk - 1) / kMChunk;
  int st0 = veff_stats(c);
  if (st0) return st0;
  const T pshift = (T)(c->vmean - c->sigma_k[ik]);
  const size_t vb = (size_t)nb * npw * sizeof(cplx<T>);
  const bool f64 = sizeof(T) == 8;
  const char* names[6] = {"mr_zn", "mr_v", "mr_vo", "mr_w", "mr_wo", "mr_y"};
  cplx<T>* buf[7];
  for (int i = 0; i < 6; ++i) {
    std::string nm = std::string(names[i]) + (f64 ? "64" : "32");
    buf[i] = static_cast<cplx<T>*>(ws_get(c, nm.c_str(), vb));
    if (!buf[i]) return PARO_ERR_CUDA;
  }
  buf[6] = static_cast<cplx<T>*>(ws_get(c, f64 ? "mr_az64" : "mr_az32", vb));
  double* part = static_cast<double*>(ws_get(c, "mr_part", (size_t)nb * nchunk * 2 * sizeof(double)));
  double* sc = static_cast<double*>(ws_get(c, "mr_scal", (size_t)nb * MNS * sizeof(double)));
  double* deps = static_cast<double*>(ws_get(c, "mr_eps", (size_t)nb * sizeof(double)));
  int* ib = static_cast<int*>(ws_get(c, "mr_int", (size_t)(nb * 3 + 4) * sizeof(int)));
  if (!buf[6] || !part || !sc || !deps || !ib) return PARO_ERR_CUDA;
  cplx<T>*zn = buf[0], *v = buf[1], *vo = buf[2], *w = buf[3], *wo = buf[4], *y = buf[5], *az = buf[6];
  int *active = ib, *its = ib + nb, *still = ib + 2 * nb, *flags = ib + 3 * nb;  // flags: nactive, bad
  const dim3 gv(nchunk, nb);
  const int tb = (nb + 127) / 128;
  const T* kin = kin_of_b<T>(B);
  if ((st0 = h2d_async(c, "mr_eps", deps, eps, nb * sizeof(double)))) return st0;
  PARO_CU(c, cudaMemsetAsync(flags, 0, 2 * sizeof(int), c->stream));
  // v_1 = P b, z_1 = P D v_1, gamma_1 = sqrt(<z_1, v_1>)
  k_mr_rhs<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, psi, hpsi, deps, v, part);
  PARO_LAUNCH(c, "k_mr_rhs");
  k_mr_band_c<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, nullptr, sc);
  PARO_LAUNCH(c, "k_mr_band_c");
  k_mr_proj_prec<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, nb, psi, v, 1, y, kin, pshift, sc, nullptr, part);
  PARO_LAUNCH(c, "k_mr_proj_prec");
  k_mr_band_c<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, nullptr, sc);
  PARO_LAUNCH(c, "k_mr_band_c");
  k_mr_zproj<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, nb, psi, y, v, sc, nullptr, part);
  PARO_LAUNCH(c, "k_mr_zproj");
  k_mr_band_start<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, sc, active, its, flags);
  PARO_LAUNCH(c, "k_mr_band_start");
  PARO_CU(c, cudaMemcpyAsync(zn, y, vb, cudaMemcpyDeviceToDevice, c->stream));
  k_mr_init_vectors<T><<<gv, kMT, 0, c->stream>>>(npw, nb, sc, zn, e, w, wo, vo);
  PARO_LAUNCH(c, "k_mr_init_vectors");
  int hflags[2] = {0, 0};
  PARO_CU(c, cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  int st;
  for (int it = 0; it < max_it && hflags[0] > 0; ++it) {
    if ((st = apply_h<T>(c, ik, nb, zn, az, 0.0, active))) return st;
    cudaEvent_t ev = prof_begin(c);
    k_mr_shift<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, psi, zn, az, deps, active, part);
    PARO_LAUNCH(c, "k_mr_shift");
    k_mr_band_c<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, active, sc);
    PARO_LAUNCH(c, "k_mr_band_c");
    k_mr_delta<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, nb, psi, zn, az, sc, active, part);
    PARO_LAUNCH(c, "k_mr_delta");
    k_mr_band_delta<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, active, sc);
    PARO_LAUNCH(c, "k_mr_band_delta");
    k_mr_lanczos<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, nb, psi, az, v, vo, y, kin, pshift, sc, active, part);
    PARO_LAUNCH(c, "k_mr_lanczos");
    std::swap(v, vo);  // v holds v_{j+1}, vo v_j (bands that stopped keep no further use of either)
    k_mr_band_c<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, active, sc);
    PARO_LAUNCH(c, "k_mr_band_c");
    k_mr_zproj<T><<<gv, kMT, 0, c->stream>>>(npw, nchunk, nb, psi, y, v, sc, active, part);
    PARO_LAUNCH(c, "k_mr_zproj");
    PARO_CU(c, cudaMemsetAsync(flags, 0, sizeof(int), c->stream));
    k_mr_band_givens<<<tb, 128, 0, c->stream>>>(nb, nchunk, part, rel_tol, active, sc, its, still, flags, flags + 1);
    PARO_LAUNCH(c, "k_mr_band_givens");
    k_mr_update<T><<<gv, kMT, 0, c->stream>>>(npw, nb, zn, y, w, wo, e, sc, active);
    PARO_LAUNCH(c, "k_mr_update");
    std::swap(w, wo);  // w holds w_{j+1}, wo w_j
    prof_end(c, f64 ? "minres_vector<f64>" : "minres_vector<f32>", ev);
    PARO_CU(c, cudaMemcpyAsync(active, still, nb * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
    PARO_CU(c, cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PARO_CU(c, cudaStreamSynchronize(c->stream));
    if (hflags[1])
      return fail(c, PARO_ERR_BREAKDOWN, "MINRES breakdown (non-finite Lanczos or Givens scalar) in orbital " +
                                             std::to_string(hflags[1] - 1));
  }
  if (iters) {
    PARO_CU(c, cudaMemcpyAsync(iters, its, nb * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PARO_CU(c, cudaStreamSynchronize(c->stream));
  }
  return PARO_OK;
}

template int minres_run<double>(Ctx*, int, int, const double2*, const double2*, const double*, double2*, double,
                                int, int*);
template int minres_run<float>(Ctx*, int, int, const float2*, const float2*, const double*, float2*, double, int,
                               int*);

}  // namespace paro
