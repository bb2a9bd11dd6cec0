// Setup and SCF kernels: twiddle tables, full-grid 3D FFT, structure factors, local pseudopotential,
// Kleinman-Bylander projectors, effective potential (Hartree + LDA-PZ), density, Pulay mixing,
// energy terms and the Ewald energy (Section 2.1, Section 2.2, Section 2.3).
#include <cmath>
#include <vector>

#include "paro_ctx.h"

namespace paro {

static const double kPi = 3.14159265358979323846;

__device__ __forceinline__ int signed_index(int j, int n) { return 2 * j < n ? j : j - n; }

// ------------------------------------------------------------------------------------------------
// twiddles exp(-2 pi i j / n)
// ------------------------------------------------------------------------------------------------
__global__ void k_twiddle(int n, double2* __restrict__ t64, float2* __restrict__ t32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s, c;
  sincospi(2.0 * (double)j / (double)n, &s, &c);
  t64[j] = make_double2(c, -s);
  t32[j] = make_float2((float)c, (float)-s);
}

int build_twiddles(Ctx* c) {
  for (int ax = 0; ax < 3; ++ax) {
    const int n = c->N[ax];
    PARO_CU(c, cudaMalloc(&c->d_tw64[ax], n * sizeof(double2)));
    PARO_CU(c, cudaMalloc(&c->d_tw32[ax], n * sizeof(float2)));
    k_twiddle<<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->d_tw64[ax], c->d_tw32[ax]);
    PARO_LAUNCH(c, "k_twiddle");
  }
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// full-grid 3D FFT (FP64), in place, unnormalised; C order (x, y, z)
// ------------------------------------------------------------------------------------------------
static const int kLB = 16;  // lines per CTA

template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_fft_z(cplx<T>* __restrict__ data, int nlines, FftPlan p,
                                               const cplx<T>* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, ls = n + 1;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* lines = tw + n;
  const int l0 = blockIdx.x * kLB, nl = min(kLB, nlines - l0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
    const int l = i / n, j = i - l * n;
    lines[l * ls + j] = data[(size_t)(l0 + l) * n + j];
  }
  __syncthreads();
  fft_lines<T, INV, false>(lines, p, nl, 1, LinesDirect{ls}, tw);
  for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
    const int l = i / n, j = i - l * n;
    data[(size_t)(l0 + l) * n + j] = lines[l * ls + j];
  }
}

// lines along an axis of element stride es; a CTA takes 16 consecutive z positions of one outer index
template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_fft_strided(cplx<T>* __restrict__ data, FftPlan p, int es, int os,
                                                     int ninner, const cplx<T>* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, ls = n + 1;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* lines = tw + n;
  const int z0 = blockIdx.x * kLB, nz = min(kLB, ninner - z0);
  const size_t base = (size_t)blockIdx.y * os + z0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < nz * n; i += blockDim.x) {
    const int l = i % nz, j = i / nz;
    lines[l * ls + j] = data[base + (size_t)j * es + l];
  }
  __syncthreads();
  fft_lines<T, INV, false>(lines, p, nz, 1, LinesDirect{ls}, tw);
  for (int i = threadIdx.x; i < nz * n; i += blockDim.x) {
    const int l = i % nz, j = i / nz;
    data[base + (size_t)j * es + l] = lines[l * ls + j];
  }
}

template <typename T, bool INV>
static int fft3d_dir(Ctx* c, cplx<T>* data) {
  const int N1 = c->N[0], N2 = c->N[1], N3 = c->N[2];
  const size_t eb = sizeof(cplx<T>);
  const size_t smz = (size_t)(N3 + kLB * (N3 + 1)) * eb;
  const size_t smy = (size_t)(N2 + kLB * (N2 + 1)) * eb;
  const size_t smx = (size_t)(N1 + kLB * (N1 + 1)) * eb;
  const cplx<T>* const* tw;
  if constexpr (sizeof(T) == 8) tw = c->d_tw64;
  else tw = c->d_tw32;
  PARO_CU(c, cudaFuncSetAttribute(k_fft_z<T, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  PARO_CU(c, cudaFuncSetAttribute(k_fft_strided<T, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  cudaEvent_t ev = prof_begin(c);
  k_fft_z<T, INV><<<(N1 * N2 + kLB - 1) / kLB, 256, smz, c->stream>>>(data, N1 * N2, c->plan[2], tw[2]);
  k_fft_strided<T, INV><<<dim3((N3 + kLB - 1) / kLB, N1), 256, smy, c->stream>>>(data, c->plan[1], N3, N2 * N3, N3,
                                                                               tw[1]);
  k_fft_strided<T, INV><<<dim3((N3 + kLB - 1) / kLB, N2), 256, smx, c->stream>>>(data, c->plan[0], N2 * N3, N3, N3,
                                                                               tw[0]);
  PARO_LAUNCH(c, "fft3d");
  prof_end(c, sizeof(T) == 8 ? "fft3d<f64>" : "fft3d<f32>", ev);
  return PARO_OK;
}

template <typename T>
int fft3d(Ctx* c, cplx<T>* data, bool inverse) {
  return inverse ? fft3d_dir<T, true>(c, data) : fft3d_dir<T, false>(c, data);
}
template int fft3d<double>(Ctx*, double2*, bool);
template int fft3d<float>(Ctx*, float2*, bool);

// ------------------------------------------------------------------------------------------------
// structure-factor phase tables: ph[a][I][j] = exp(-i 2 pi n f_{I,a}), n = signed grid index j
// ------------------------------------------------------------------------------------------------
__global__ void k_phase_tables(int nat, int N1, int N2, int N3, const double* __restrict__ frac,
                               double2* __restrict__ ph) {
  const int tot = N1 + N2 + N3;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nat * tot) return;
  const int I = idx / tot;
  int j = idx - I * tot, a = 0, n = N1;
  if (j >= N1) { j -= N1; a = 1; n = N2; if (j >= N2) { j -= N2; a = 2; n = N3; } }
  const int s = signed_index(j, n);
  double sn, cs;
  sincospi(2.0 * (double)s * frac[I * 3 + a], &sn, &cs);
  ph[idx] = make_double2(cs, -sn);
}

static double2* phase_tables(Ctx* c) {
  const int tot = c->N[0] + c->N[1] + c->N[2];
  double2* ph = static_cast<double2*>(ws_get(c, "phase_tables", (size_t)c->nat * tot * sizeof(double2)));
  double* dfrac = static_cast<double*>(ws_get(c, "frac", (size_t)c->nat * 3 * sizeof(double)));
  if (!ph || !dfrac) return nullptr;
  // fractional coordinates f_a = R . b_a / (2 pi)
  std::vector<double> frac(c->nat * 3);
  for (int I = 0; I < c->nat; ++I)
    for (int a = 0; a < 3; ++a) {
      double s = 0;
      for (int x = 0; x < 3; ++x) s += c->pos[I * 3 + x] * c->bmat[a * 3 + x];
      frac[I * 3 + a] = s / (2.0 * kPi);
    }
  if (cudaMemcpyAsync(dfrac, frac.data(), frac.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess) {
    fail(c, PARO_ERR_CUDA, "phase table copy failed");
    return nullptr;
  }
  k_phase_tables<<<(c->nat * tot + 255) / 256, 256, 0, c->stream>>>(c->nat, c->N[0], c->N[1], c->N[2], dfrac, ph);
  if (cudaGetLastError() != cudaSuccess) {
    fail(c, PARO_ERR_CUDA, "k_phase_tables launch failed");
    return nullptr;
  }
  return ph;
}

struct Mat3 {
  double m[9];
};

// ------------------------------------------------------------------------------------------------
// local pseudopotential V_loc(G) on the density sphere, then V_loc(r) by an inverse FFT
// ------------------------------------------------------------------------------------------------
__global__ void k_vloc_g(int N1, int N2, int N3, Mat3 B, double ecut4, double Z, double rc, double A, double a,
                         double omega, int nat, const double2* __restrict__ ph, double2* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int ng = N1 * N2 * N3;
  if (idx >= ng) return;
  const int j3 = idx % N3, j2 = (idx / N3) % N2, j1 = idx / (N2 * N3);
  const int n1 = signed_index(j1, N1), n2 = signed_index(j2, N2), n3 = signed_index(j3, N3);
  const double gx = n1 * B.m[0] + n2 * B.m[3] + n3 * B.m[6];
  const double gy = n1 * B.m[1] + n2 * B.m[4] + n3 * B.m[7];
  const double gz = n1 * B.m[2] + n2 * B.m[5] + n3 * B.m[8];
  const double g2 = gx * gx + gy * gy + gz * gz;
  double2 v = make_double2(0.0, 0.0);
  if (0.5 * g2 <= ecut4 && 2 * abs(n1) < N1 && 2 * abs(n2) < N2 && 2 * abs(n3) < N3) {
    const int tot = N1 + N2 + N3;
    double2 sf = make_double2(0.0, 0.0);
    for (int I = 0; I < nat; ++I) {
      const double2* p = ph + (size_t)I * tot;
      sf = cadd(sf, cmul(cmul(p[j1], p[N1 + j2]), p[N1 + N2 + j3]));
    }
    double form = A * pow(kPi, 1.5) * a * a * a * exp(-g2 * a * a / 4.0);
    form += g2 > 0.0 ? -4.0 * kPi * Z * exp(-g2 * rc * rc / 4.0) / g2 : kPi * Z * rc * rc;
    v = cscale(sf, form / omega);
  }
  out[idx] = v;
}

__global__ void k_real_part(int n, const double2* __restrict__ z, double* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = z[i].x;
}

int build_vloc(Ctx* c) {
  double2* ph = phase_tables(c);
  if (!ph) return PARO_ERR_CUDA;
  double2* vg = static_cast<double2*>(ws_get(c, "grid_c0", (size_t)c->ngrid * sizeof(double2)));
  if (!vg) return PARO_ERR_CUDA;
  Mat3 B;
  for (int i = 0; i < 9; ++i) B.m[i] = c->bmat[i];
  k_vloc_g<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->N[0], c->N[1], c->N[2], B, 4.0 * c->ecut, c->Z, c->rc,
                                                          c->A, c->a, c->omega, c->nat, ph, vg);
  PARO_LAUNCH(c, "k_vloc_g");
  int st = fft3d<double>(c, vg, true);
  if (st) return st;
  if (!c->d_vloc) PARO_CU(c, cudaMalloc(&c->d_vloc, (size_t)c->ngrid * sizeof(double)));
  k_real_part<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, vg, c->d_vloc);
  PARO_LAUNCH(c, "k_real_part");
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// dL/dR_I through V_loc (adjoint of H psi): with V_loc(r) = sum_G V_loc(G) exp(i G.r) and
// dV_loc(G)/dR_Ia = -i G_a Omega^{-1} exp(-i G.R_I) v(G),
//   dL/dR_Ia = Re sum_G (-i G_a) Omega^{-1} v(G) exp(-i G.R_I) conj(g^(G)),  g^ = forward DFT of dL/dV(r).
// k_vloc_weight: wg(G) = Omega^{-1} v(G) conj(g^(G)) on the V_loc support, 0 elsewhere (in place).
// k_vloc_force: one CTA per (atom, grid chunk), partial sums per chunk; k_vloc_force_reduce sums the
// chunks in a fixed order.
// ------------------------------------------------------------------------------------------------
__global__ void k_to_complex(int n, const double* __restrict__ r, double2* __restrict__ z);

__global__ void k_vloc_weight(int N1, int N2, int N3, Mat3 B, double ecut4, double Z, double rc, double A, double a,
                              double omega, double2* __restrict__ g) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N1 * N2 * N3) return;
  const int j3 = idx % N3, j2 = (idx / N3) % N2, j1 = idx / (N2 * N3);
  const int n1 = signed_index(j1, N1), n2 = signed_index(j2, N2), n3 = signed_index(j3, N3);
  const double gx = n1 * B.m[0] + n2 * B.m[3] + n3 * B.m[6];
  const double gy = n1 * B.m[1] + n2 * B.m[4] + n3 * B.m[7];
  const double gz = n1 * B.m[2] + n2 * B.m[5] + n3 * B.m[8];
  const double g2 = gx * gx + gy * gy + gz * gz;
  double2 out = make_double2(0.0, 0.0);
  if (0.5 * g2 <= ecut4 && 2 * abs(n1) < N1 && 2 * abs(n2) < N2 && 2 * abs(n3) < N3) {
    double form = A * pow(kPi, 1.5) * a * a * a * exp(-g2 * a * a / 4.0);
    form += g2 > 0.0 ? -4.0 * kPi * Z * exp(-g2 * rc * rc / 4.0) / g2 : kPi * Z * rc * rc;
    out = cscale(cconj(g[idx]), form / omega);
  }
  g[idx] = out;
}

__global__ void __launch_bounds__(256) k_vloc_force(int N1, int N2, int N3, Mat3 B, int chunk,
                                                    const double2* __restrict__ ph, const double2* __restrict__ wg,
                                                    double* __restrict__ part) {
  __shared__ double red[32];
  const int I = blockIdx.y, tot = N1 + N2 + N3, ng = N1 * N2 * N3;
  const double2* p = ph + (size_t)I * tot;
  const int i0 = blockIdx.x * chunk, i1 = min(ng, i0 + chunk);
  double f[3] = {0.0, 0.0, 0.0};
  for (int idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x) {
    const double2 w = wg[idx];
    if (w.x == 0.0 && w.y == 0.0) continue;
    const int j3 = idx % N3, j2 = (idx / N3) % N2, j1 = idx / (N2 * N3);
    const int n1 = signed_index(j1, N1), n2 = signed_index(j2, N2), n3 = signed_index(j3, N3);
    const double2 sw = cmul(cmul(cmul(p[j1], p[N1 + j2]), p[N1 + N2 + j3]), w);  // exp(-i G.R_I) wg
    // Re[(-i G_a) sw] = G_a Im(sw)
    for (int al = 0; al < 3; ++al) f[al] += (n1 * B.m[al] + n2 * B.m[3 + al] + n3 * B.m[6 + al]) * sw.y;
  }
  for (int al = 0; al < 3; ++al) {
    const double v = block_sum(f[al], red);
    if (threadIdx.x == 0) part[((size_t)I * gridDim.x + blockIdx.x) * 3 + al] = v;
  }
}

__global__ void k_vloc_force_reduce(int nat, int nchunk, const double* __restrict__ part, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nat * 3) return;
  const int I = i / 3, al = i - 3 * I;
  double s = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) s += part[((size_t)I * nchunk + ch) * 3 + al];
  out[i] = s;
}

int vloc_position_grad(Ctx* c, const double* gv, double* gpos) {
  if (c->nat == 0) return PARO_OK;
  double2* ph = phase_tables(c);
  double2* g = static_cast<double2*>(ws_get(c, "grid_c1", (size_t)c->ngrid * sizeof(double2)));
  const int chunk = 4096, nchunk = (c->ngrid + chunk - 1) / chunk;
  double* part = static_cast<double*>(ws_get(c, "vforce_part", (size_t)c->nat * nchunk * 3 * sizeof(double)));
  if (!ph || !g || !part) return PARO_ERR_CUDA;
  k_to_complex<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, gv, g);
  PARO_LAUNCH(c, "k_to_complex");
  int st = fft3d<double>(c, g, false);
  if (st) return st;
  Mat3 B;
  for (int i = 0; i < 9; ++i) B.m[i] = c->bmat[i];
  k_vloc_weight<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->N[0], c->N[1], c->N[2], B, 4.0 * c->ecut, c->Z,
                                                               c->rc, c->A, c->a, c->omega, g);
  PARO_LAUNCH(c, "k_vloc_weight");
  k_vloc_force<<<dim3(nchunk, c->nat), 256, 0, c->stream>>>(c->N[0], c->N[1], c->N[2], B, chunk, ph, g, part);
  PARO_LAUNCH(c, "k_vloc_force");
  k_vloc_force_reduce<<<(c->nat * 3 + 127) / 128, 128, 0, c->stream>>>(c->nat, nchunk, part, gpos);
  PARO_LAUNCH(c, "k_vloc_force_reduce");
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Kleinman-Bylander projector table beta[4 I + j][g], j = s, px, py, pz
// ------------------------------------------------------------------------------------------------
__global__ void k_beta(int npw, int nat, int N1, int N2, int N3, Mat3 B, double kx, double ky, double kz,
                       const int* __restrict__ miller, const double2* __restrict__ ph,
                       const double2* __restrict__ kph, double rc, double omega, double2* __restrict__ beta,
                       float2* __restrict__ beta32) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = blockIdx.y;
  if (g >= npw) return;
  const int n1 = miller[3 * g], n2 = miller[3 * g + 1], n3 = miller[3 * g + 2];
  const double qx = kx + n1 * B.m[0] + n2 * B.m[3] + n3 * B.m[6];
  const double qy = ky + n1 * B.m[1] + n2 * B.m[4] + n3 * B.m[7];
  const double qz = kz + n1 * B.m[2] + n2 * B.m[5] + n3 * B.m[8];
  const double q2 = qx * qx + qy * qy + qz * qz;
  const double gauss = exp(-q2 * rc * rc / 4.0);
  const double pi15 = pow(kPi, 1.5);
  const double n0 = 1.0 / sqrt(pow(kPi / 2.0, 1.5) * rc * rc * rc);
  const double nn1 = 1.0 / sqrt(pow(kPi / 2.0, 1.5) * pow(rc, 5.0) / 4.0);
  const double fs = n0 * pi15 * rc * rc * rc * gauss;
  const double fp = nn1 * pi15 * pow(rc, 5.0) / 2.0 * gauss;  // p~_a = -i fp q_a
  const int tot = N1 + N2 + N3;
  const double2* p = ph + (size_t)I * tot;
  const int j1 = n1 < 0 ? n1 + N1 : n1, j2 = n2 < 0 ? n2 + N2 : n2, j3 = n3 < 0 ? n3 + N3 : n3;
  double2 phase = cmul(cmul(cmul(p[j1], p[N1 + j2]), p[N1 + N2 + j3]), kph[I]);
  phase = cscale(phase, 1.0 / sqrt(omega));
  const double2 vs = cscale(phase, fs);
  const double2 mi = make_double2(phase.y, -phase.x);  // -i * phase
  const double2 vx = cscale(mi, fp * qx), vy = cscale(mi, fp * qy), vz = cscale(mi, fp * qz);
  const size_t row = (size_t)4 * I;
  beta[(row + 0) * npw + g] = vs;
  beta[(row + 1) * npw + g] = vx;
  beta[(row + 2) * npw + g] = vy;
  beta[(row + 3) * npw + g] = vz;
  beta32[(row + 0) * npw + g] = make_float2((float)vs.x, (float)vs.y);
  beta32[(row + 1) * npw + g] = make_float2((float)vx.x, (float)vx.y);
  beta32[(row + 2) * npw + g] = make_float2((float)vy.x, (float)vy.y);
  beta32[(row + 3) * npw + g] = make_float2((float)vz.x, (float)vz.y);
}

int build_beta(Ctx* c) {
  double2* ph = phase_tables(c);
  if (!ph) return PARO_ERR_CUDA;
  Mat3 B;
  for (int i = 0; i < 9; ++i) B.m[i] = c->bmat[i];
  c->nproj = 4 * c->nat;
  double2* kph = static_cast<double2*>(ws_get(c, "kphase", (size_t)c->nat * sizeof(double2)));
  double* norms = static_cast<double*>(ws_get(c, "beta_norms", (size_t)c->nproj * sizeof(double)));
  if (!kph || !norms) return PARO_ERR_CUDA;
  c->beta_norm2_max.assign((size_t)c->nk * c->nat * 2, 0.0);
  for (int ik = 0; ik < c->nk; ++ik) {
    Basis& b = c->bases[ik];
    std::vector<double2> hk(c->nat);
    for (int I = 0; I < c->nat; ++I) {
      double kr = 0;
      for (int x = 0; x < 3; ++x) kr += b.kcart[x] * c->pos[I * 3 + x];
      hk[I] = make_double2(std::cos(kr), -std::sin(kr));
    }
    PARO_CU(c, cudaMemcpyAsync(kph, hk.data(), c->nat * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    if (!b.d_beta) {
      PARO_CU(c, cudaMalloc(&b.d_beta, (size_t)c->nproj * b.npw * sizeof(double2)));
      PARO_CU(c, cudaMalloc(&b.d_beta32, (size_t)c->nproj * b.npw * sizeof(float2)));
    }
    for (float4** img : {&b.d_beta_img_cn, &b.d_beta_img_wx}) {  // formed again from the new projectors
      if (*img) {
        PARO_CU(c, cudaStreamSynchronize(c->stream));
        cudaFree(*img);
        *img = nullptr;
      }
    }
    k_beta<<<dim3((b.npw + 127) / 128, c->nat), 128, 0, c->stream>>>(b.npw, c->nat, c->N[0], c->N[1], c->N[2], B,
                                                                    b.kcart[0], b.kcart[1], b.kcart[2], b.d_miller,
                                                                    ph, kph, c->kb_rc, c->omega, b.d_beta,
                                                                    b.d_beta32);
    PARO_LAUNCH(c, "k_beta");
    int st = band_norms<double>(c, c->nproj, b.npw, b.d_beta, b.npw, norms);
    if (st) return st;
    std::vector<double> h(c->nproj);
    PARO_CU(c, cudaMemcpyAsync(h.data(), norms, c->nproj * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PARO_CU(c, cudaStreamSynchronize(c->stream));
    for (int I = 0; I < c->nat; ++I) {
      double* m = &c->beta_norm2_max[((size_t)ik * c->nat + I) * 2];
      m[0] = h[4 * I];
      m[1] = std::max(h[4 * I + 1], std::max(h[4 * I + 2], h[4 * I + 3]));
    }
  }
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// effective potential on the grid: plane-major copies scaled by 1/N_grid, min and mean
// ------------------------------------------------------------------------------------------------
__global__ void k_vplane(int N1, int N2, int N3, const double* __restrict__ v, double* __restrict__ vp,
                         float* __restrict__ vp32, double inv_n) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over the plane-major output
  if (idx >= N1 * N2 * N3) return;
  const int y = idx % N2, x = (idx / N2) % N1, z = idx / (N1 * N2);
  const double val = v[((size_t)x * N2 + y) * N3 + z] * inv_n;
  vp[idx] = val;
  vp32[idx] = (float)val;
}

// sum and minimum of V over the grid: per-CTA partials over fixed chunks, then one CTA combines them
// in order (deterministic)
__global__ void k_min_sum(int n, const double* __restrict__ v, double* __restrict__ part) {
  __shared__ double red[32];
  __shared__ double rmin[32];
  double s = 0.0, mn = 1e300;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s += v[i];
    mn = fmin(mn, v[i]);
  }
  s = block_sum(s, red);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) rmin[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mn = fmin(mn, rmin[w]);
    part[2 * blockIdx.x] = s;
    part[2 * blockIdx.x + 1] = fmin(mn, rmin[0]);
  }
}

// one warp: lane-strided partial sums and minima, then a fixed-order shuffle tree (a single thread's
// chain of dependent FP64 adds would cost ~100 cycles per block here)
__global__ void k_min_sum_final(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  const int lane = threadIdx.x;
  double s = 0.0, mn = 1e300;
  for (int b = lane; b < nblk; b += 32) {
    s += part[2 * b];
    mn = fmin(mn, part[2 * b + 1]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if (lane == 0) {
    out[0] = s;
    out[1] = mn;
  }
}

int set_veff_device(Ctx* c, const double* v_dev) {
  if (!c->d_veff) {
    PARO_CU(c, cudaMalloc(&c->d_veff, (size_t)c->ngrid * sizeof(double)));
    PARO_CU(c, cudaMalloc(&c->d_vplane, (size_t)c->ngrid * sizeof(double)));
    PARO_CU(c, cudaMalloc(&c->d_vplane32, (size_t)c->ngrid * sizeof(float)));
  }
  if (v_dev != c->d_veff)
    PARO_CU(c, cudaMemcpyAsync(c->d_veff, v_dev, (size_t)c->ngrid * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
  k_vplane<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->N[0], c->N[1], c->N[2], c->d_veff, c->d_vplane,
                                                          c->d_vplane32, 1.0 / c->ngrid);
  PARO_LAUNCH(c, "k_vplane");
  const int nblk = 304;
  double* ms = static_cast<double*>(ws_get(c, "vminsum", (2 + 2 * nblk) * sizeof(double)));
  if (!ms) return PARO_ERR_CUDA;
  k_min_sum<<<nblk, 256, 0, c->stream>>>(c->ngrid, c->d_veff, ms + 2);
  PARO_LAUNCH(c, "k_min_sum");
  k_min_sum_final<<<1, 32, 0, c->stream>>>(nblk, ms + 2, ms);
  PARO_LAUNCH(c, "k_min_sum_final");
  // the sum and the minimum come back without waiting for the stream; veff_stats() reads them when the
  // PCG shift is next needed
  int st = d2h_async(c, "vstats", ms, 2 * sizeof(double), nullptr);
  if (st) return st;
  c->vstats_pending = true;
  c->have_veff = true;
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Hartree and LDA-PZ
// ------------------------------------------------------------------------------------------------
__global__ void k_to_complex(int n, const double* __restrict__ r, double2* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = make_double2(r[i], 0.0);
}

// rho_g (unnormalised forward FFT of rho) -> V_H(G) = 4 pi rho(G)/G^2 with rho(G) = rho_g / N; partial
// sums of |rho(G)|^2 / G^2 per block for E_H.
// 1 / |G|^2 on the grid (0 at G = 0): the Coulomb factor of every Hartree solve, formed once per grid
__global__ void k_inv_g2(int N1, int N2, int N3, Mat3 B, double* __restrict__ ig2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N1 * N2 * N3) return;
  const int j3 = idx % N3, j2 = (idx / N3) % N2, j1 = idx / (N2 * N3);
  const int n1 = signed_index(j1, N1), n2 = signed_index(j2, N2), n3 = signed_index(j3, N3);
  const double gx = n1 * B.m[0] + n2 * B.m[3] + n3 * B.m[6];
  const double gy = n1 * B.m[1] + n2 * B.m[4] + n3 * B.m[7];
  const double gz = n1 * B.m[2] + n2 * B.m[5] + n3 * B.m[8];
  const double g2 = gx * gx + gy * gy + gz * gz;
  ig2[idx] = g2 > 0.0 ? 1.0 / g2 : 0.0;
}

// V_H(G) = 4 pi rho(G) / |G|^2 in place (rho(G) = z / N_grid), and per block partials of |rho(G)|^2 / |G|^2
__global__ void k_hartree_tab(int ng, const double* __restrict__ ig2, double2* __restrict__ z,
                              double* __restrict__ part) {
  __shared__ double red[32];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (idx < ng) {
    const double f = ig2[idx];
    const double2 r = cscale(z[idx], 1.0 / ng);
    e = (r.x * r.x + r.y * r.y) * f;
    z[idx] = cscale(r, 4.0 * kPi * f);
  }
  e = block_sum(e, red);
  if (threadIdx.x == 0) part[blockIdx.x] = e;
}


// Perdew-Zunger LDA exchange-correlation energy per electron and potential at density rho, in R
// (double, or float where the potential only enters FP32 H psi and the energy sums stay FP64)
template <typename R>
__device__ __forceinline__ void lda_pz(R rho, R* eps, R* v) {
  if (!(rho >= (R)1e-30)) { *eps = 0; *v = 0; return; }
  const R pi = (R)kPi;
  const R ex = (R)-0.75 * cbrt((R)3 * rho / pi);
  const R vx = (R)4 / (R)3 * ex;
  const R rs = cbrt((R)3 / ((R)4 * pi * rho));
  R ec, vc;
  if (rs >= (R)1) {
    const R s = sqrt(rs);
    const R den = (R)1 + (R)1.0529 * s + (R)0.3334 * rs;
    ec = (R)-0.1423 / den;
    vc = ec * ((R)1 + (R)7 / (R)6 * (R)1.0529 * s + (R)4 / (R)3 * (R)0.3334 * rs) / den;
  } else {
    const R lr = log(rs);
    ec = (R)0.0311 * lr - (R)0.048 + (R)0.0020 * rs * lr - (R)0.0116 * rs;
    vc = (R)0.0311 * lr + ((R)-0.048 - (R)0.0311 / (R)3) + (R)2 / (R)3 * (R)0.0020 * rs * lr +
         ((R)2 * (R)-0.0116 - (R)0.0020) / (R)3 * rs;
  }
  *eps = ex + ec;
  *v = vx + vc;
}

// eps_xc of the same functional in FP64 accuracy with a fraction of the FP64 instructions (the energy's
// grid sum; GB300's FP64 pipe makes CUDA's FP64 cube root the cost of that pass): the cube root of rho, its
// reciprocal, the square root of r_s and the reciprocal of the correlation denominator each start from an
// FP32 estimate and take one Newton step in FP64, which squares the estimate's ~1e-7 relative error; the
// high-density branch keeps the FP64 logarithm.
__device__ __forceinline__ double lda_pz_eps64(double rho) {
  if (!(rho >= 1e-30)) return 0.0;
  const float c0f = cbrtf((float)rho);
  const double c0 = c0f;
  const double c = fma(fma(-c0 * c0, c0, rho), (double)(1.0f / (3.0f * c0f * c0f)), c0);  // rho^(1/3)
  const double i0 = (double)(1.0f / c0f);
  const double ic = fma(i0, fma(-c, i0, 1.0), i0);  // 1 / c
  const double ex = -0.75 * 0.9847450218426965 * c;  // -(3/4) (3 rho / pi)^(1/3)
  const double rs = 0.6203504908994001 * ic;         // (3 / (4 pi rho))^(1/3)
  double ec;
  if (rs >= 1.0) {
    const float s0f = sqrtf((float)rs);
    const double s0 = s0f;
    const double sq = fma(fma(-s0, s0, rs), (double)(0.5f / s0f), s0);
    const double den = fma(0.3334, rs, fma(1.0529, sq, 1.0));
    const double d0 = (double)(1.0f / (float)den);
    ec = -0.1423 * fma(d0, fma(-den, d0, 1.0), d0);
  } else {
    const double lr = log(rs);
    ec = 0.0311 * lr - 0.048 + 0.0020 * rs * lr - 0.0116 * rs;
  }
  return ex + ec;
}

template <typename R>
__global__ void k_veff_combine(int n, const double* __restrict__ vloc, const double2* __restrict__ vh,
                               const double* __restrict__ rho, double* __restrict__ veff) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R e, v;
  lda_pz<R>((R)rho[i], &e, &v);
  veff[i] = vloc[i] + vh[i].x + (double)v;
}

static int sum_parts(Ctx* c, const double* part, int n, double* out) {
  std::vector<double> h(n);
  PARO_CU(c, cudaMemcpyAsync(h.data(), part, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  double s = 0;
  for (int i = 0; i < n; ++i) s += h[i];
  *out = s;
  return PARO_OK;
}

static const double* inv_g2_table(Ctx* c);

// Partial sums of E_H of rho (hartree_blocks(c) doubles in part; E_H = 2 pi Omega times their sum) and,
// when potential, V_H(r) in z (real parts). Launches only: the energy alone needs only the forward FFT
// and no host synchronisation until the caller reads the partials.
static int hartree_blocks(const Ctx* c) { return (c->ngrid + 255) / 256; }
// ------------------------------------------------------------------------------------------------
// Hartree energy of the real density from one half-length transform: the even and odd z planes packed as
// the real and imaginary parts of one complex array on the (N1, N2, M = N3/2) grid, transformed, then
// unpacked with k = (kx, ky, kz), kz < M, and -k taken modulo (N1, N2, M):
//   A(k) = (Z(k) + conj Z(-k)) / 2,  B(k) = (Z(k) - conj Z(-k)) / (2i)   (the transforms of the even and odd
//   planes), rho(kx, ky, kz) = A(k) + W^kz B(k), rho(kx, ky, kz + M) = A(k) - W^kz B(k), W = exp(-2 pi i / N3).
// The same coefficients as the full complex transform, for half its work on GB300's slow FP64 pipe.
// ------------------------------------------------------------------------------------------------
__global__ void k_pack_even_odd(int n, int M, const double* __restrict__ rho, double2* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over nxy * M
  if (i >= n) return;
  const int xy = i / M, m = i - xy * M;
  const double* r = rho + (size_t)xy * 2 * M + 2 * m;
  z[i] = make_double2(r[0], r[1]);
}

// per-CTA partial sums of |rho(G)|^2 / |G|^2 over both G of each half-grid point (the layout of
// k_hartree_tab's partials: one per 256 full-grid points, the CTAs beyond the half grid write zero)
__global__ void k_hartree_half(int N1, int N2, int M, const double* __restrict__ ig2, const double2* __restrict__ z,
                               const double2* __restrict__ tw3, double* __restrict__ part) {
  __shared__ double red[32];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nh = N1 * N2 * M, N3 = 2 * M;
  double e = 0.0;
  if (idx < nh) {
    const int kx = idx / (N2 * M), rem = idx - kx * (N2 * M), ky = rem / M, km = rem - ky * M;
    const int nkx = kx ? N1 - kx : 0, nky = ky ? N2 - ky : 0, nkm = km ? M - km : 0;
    const double2 zk = z[idx], zn = cconj(z[((size_t)nkx * N2 + nky) * M + nkm]);
    const double2 a = cscale(cadd(zk, zn), 0.5);
    const double2 d = csub(zk, zn);
    const double2 b = make_double2(0.5 * d.y, -0.5 * d.x);  // d / (2i)
    const double2 wb = cmul(tw3[km], b);                      // tw3[j] = exp(-2 pi i j / N3)
    const double inv = 1.0 / ((double)N1 * N2 * N3);
    const double2 r1 = cscale(cadd(a, wb), inv), r2 = cscale(csub(a, wb), inv);
    const size_t base = ((size_t)kx * N2 + ky) * N3 + km;
    e = ig2[base] * (r1.x * r1.x + r1.y * r1.y) + ig2[base + M] * (r2.x * r2.x + r2.y * r2.y);
  }
  e = block_sum(e, red);
  if (threadIdx.x == 0) part[blockIdx.x] = e;
}

// the N3/2-point FP64 twiddle table (built once per grid)
static const double2* half_twiddles(Ctx* c) {
  const int M = c->N[2] / 2;
  double2* t64 = static_cast<double2*>(ws_get(c, "tw64_half", (size_t)M * sizeof(double2)));
  float2* t32 = static_cast<float2*>(ws_get(c, "tw32_half", (size_t)M * sizeof(float2)));
  if (!t64 || !t32) return nullptr;
  if (!c->have_tw_half) {
    k_twiddle<<<(M + 127) / 128, 128, 0, c->stream>>>(M, t64, t32);
    if (cudaGetLastError() != cudaSuccess) return nullptr;
    c->have_tw_half = true;
  }
  return t64;
}

// forward transform (FP64, unnormalised) of the (N1, N2, N3/2) grid in z
static int fft3d_half_fwd(Ctx* c, double2* z) {
  const int N1 = c->N[0], N2 = c->N[1], M = c->N[2] / 2;
  const double2* twh = half_twiddles(c);
  if (!twh) return fail(c, PARO_ERR_CUDA, "hartree: half-length twiddles");
  const FftPlan ph = fft_plan(M);
  const size_t eb = sizeof(double2);
  const size_t smz = (size_t)(M + kLB * (M + 1)) * eb;
  const size_t smy = (size_t)(N2 + kLB * (N2 + 1)) * eb;
  const size_t smx = (size_t)(N1 + kLB * (N1 + 1)) * eb;
  PARO_CU(c, cudaFuncSetAttribute(k_fft_z<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  PARO_CU(c, cudaFuncSetAttribute(k_fft_strided<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  100 * 1024));
  cudaEvent_t ev = prof_begin(c);
  k_fft_z<double, false><<<(N1 * N2 + kLB - 1) / kLB, 256, smz, c->stream>>>(z, N1 * N2, ph, twh);
  k_fft_strided<double, false><<<dim3((M + kLB - 1) / kLB, N1), 256, smy, c->stream>>>(z, c->plan[1], M, N2 * M, M,
                                                                                    c->d_tw64[1]);
  k_fft_strided<double, false><<<dim3((M + kLB - 1) / kLB, N2), 256, smx, c->stream>>>(z, c->plan[0], N2 * M, M, M,
                                                                                    c->d_tw64[0]);
  PARO_LAUNCH(c, "fft3d_half");
  prof_end(c, "fft3d<f64>", ev);
  return PARO_OK;
}

static int hartree_g(Ctx* c, const double* rho_dev, double2* z, double* part, bool potential) {
  const int nblk = hartree_blocks(c);
  if (!potential && c->N[2] % 2 == 0) {  // the energy alone: the half-length transform of the real density
    const int M = c->N[2] / 2, nh = c->N[0] * c->N[1] * M;
    k_pack_even_odd<<<(nh + 255) / 256, 256, 0, c->stream>>>(nh, M, rho_dev, z);
    PARO_LAUNCH(c, "k_pack_even_odd");
    int st = fft3d_half_fwd(c, z);
    if (st) return st;
    const double* ig2 = inv_g2_table(c);
    if (!ig2) return fail(c, PARO_ERR_CUDA, "hartree: 1/|G|^2 table");
    k_hartree_half<<<nblk, 256, 0, c->stream>>>(c->N[0], c->N[1], M, ig2, z, c->d_tw64[2], part);
    PARO_LAUNCH(c, "k_hartree_half");
    return PARO_OK;
  }
  k_to_complex<<<nblk, 256, 0, c->stream>>>(c->ngrid, rho_dev, z);
  PARO_LAUNCH(c, "k_to_complex");
  int st = fft3d<double>(c, z, false);
  if (st) return st;
  const double* ig2 = inv_g2_table(c);
  if (!ig2) return fail(c, PARO_ERR_CUDA, "hartree: 1/|G|^2 table");
  k_hartree_tab<<<nblk, 256, 0, c->stream>>>(c->ngrid, ig2, z, part);
  PARO_LAUNCH(c, "k_hartree_tab");
  if (potential && (st = fft3d<double>(c, z, true))) return st;
  return PARO_OK;
}
static double hartree_energy(const Ctx* c, double part_sum) { return 0.5 * c->omega * 4.0 * kPi * part_sum; }

// V_H(r) for the mixed path: the density's FFT, 4 pi / |G|^2 and the inverse FFT in FP32 (the potential
// enters H psi as FP32 planes); no energy.
__global__ void k_to_complex32(int n, const double* __restrict__ r, float2* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = make_float2((float)r[i], 0.f);
}
__global__ void k_hartree_pot32(int ng, const double* __restrict__ ig2, float2* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ng) z[i] = cscale(z[i], (float)(4.0 * kPi * ig2[i] / ng));
}
__global__ void k_veff_combine32(int n, const double* __restrict__ vloc, const float2* __restrict__ vh,
                                 const double* __restrict__ rho, double* __restrict__ veff) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float e, v;
  lda_pz<float>((float)rho[i], &e, &v);
  veff[i] = vloc[i] + (double)(vh[i].x + v);
}

static const double* inv_g2_table(Ctx* c) {
  double* ig2 = static_cast<double*>(ws_get(c, "inv_g2", (size_t)c->ngrid * sizeof(double)));
  if (!ig2) return nullptr;
  if (!c->have_inv_g2) {  // the cell and grid are fixed for the context's life
    Mat3 B;
    for (int i = 0; i < 9; ++i) B.m[i] = c->bmat[i];
    k_inv_g2<<<hartree_blocks(c), 256, 0, c->stream>>>(c->N[0], c->N[1], c->N[2], B, ig2);
    if (cudaGetLastError() != cudaSuccess) return nullptr;
    c->have_inv_g2 = true;
  }
  return ig2;
}

int veff_from_density(Ctx* c, const double* rho_dev, double* eh_out, double* exc_out) {
  (void)exc_out;
  if (!c->have_pp) return fail(c, PARO_ERR_STATE, "no local pseudopotential set");
  if (c->prec == PARO_MIXED && !eh_out) {
    float2* z = static_cast<float2*>(ws_get(c, "grid_c0_32", (size_t)c->ngrid * sizeof(float2)));
    double* v = static_cast<double*>(ws_get(c, "grid_r0", (size_t)c->ngrid * sizeof(double)));
    const double* ig2 = inv_g2_table(c);
    if (!z || !v || !ig2) return fail(c, PARO_ERR_CUDA, "veff_from_density: workspace");
    const int nblk = hartree_blocks(c);
    k_to_complex32<<<nblk, 256, 0, c->stream>>>(c->ngrid, rho_dev, z);
    PARO_LAUNCH(c, "k_to_complex32");
    int st = fft3d<float>(c, z, false);
    if (st) return st;
    k_hartree_pot32<<<nblk, 256, 0, c->stream>>>(c->ngrid, ig2, z);
    PARO_LAUNCH(c, "k_hartree_pot32");
    if ((st = fft3d<float>(c, z, true))) return st;
    k_veff_combine32<<<nblk, 256, 0, c->stream>>>(c->ngrid, c->d_vloc, z, rho_dev, v);
    PARO_LAUNCH(c, "k_veff_combine32");
    return set_veff_device(c, v);
  }
  double2* z = static_cast<double2*>(ws_get(c, "grid_c0", (size_t)c->ngrid * sizeof(double2)));
  double* v = static_cast<double*>(ws_get(c, "grid_r0", (size_t)c->ngrid * sizeof(double)));
  if (!z || !v) return PARO_ERR_CUDA;
  double* part = static_cast<double*>(ws_get(c, "hartree_part", (size_t)hartree_blocks(c) * sizeof(double)));
  if (!part) return PARO_ERR_CUDA;
  int st = hartree_g(c, rho_dev, z, part, true);
  if (st) return st;
  if (c->prec == PARO_MIXED)  // the potential reaches H psi as FP32 planes: V_xc in FP32 loses nothing
    k_veff_combine<float><<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, c->d_vloc, z, rho_dev, v);
  else
    k_veff_combine<double><<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, c->d_vloc, z, rho_dev, v);
  PARO_LAUNCH(c, "k_veff_combine");
  if (eh_out) {
    double sp = 0;
    if ((st = sum_parts(c, part, hartree_blocks(c), &sp))) return st;
    *eh_out = hartree_energy(c, sp);
  }
  return set_veff_device(c, v);
}

// ------------------------------------------------------------------------------------------------
// density of occupied orbitals: pass 1 (z inverse) then, per (plane, band group), the inverse plane
// FFT and sum of w |psi(r)|^2; partial planes per group are reduced in a fixed order.
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512, 1) k_plane_density(const cplx<T>* __restrict__ S, int ncol, int nbands, int gsize,
                                const int* __restrict__ col_x, const int* __restrict__ col_y,
                                const int* __restrict__ xrows, int nxr, FftPlan px, FftPlan py,
                                const cplx<T>* __restrict__ twx, const cplx<T>* __restrict__ twy, double wfac,
                                const double* __restrict__ wsq, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N1 = px.n, N2 = py.n;
  cplx<T>* tx = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* ty = tx + N1;
  cplx<T>* P = ty + N2;
  double* acc = reinterpret_cast<double*>(P + N1 * N2);
  const int z = blockIdx.x, grp = blockIdx.y, N3 = gridDim.x;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) acc[i] = 0.0;
  const int b0 = grp * gsize, b1 = min(nbands, b0 + gsize);
  for (int b = b0; b < b1; ++b) {
    for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) P[i] = mk<T>(0, 0);
    __syncthreads();
    const cplx<T>* Sz = S + ((size_t)b * N3 + z) * ncol;
    for (int cc = threadIdx.x; cc < ncol; cc += blockDim.x) P[col_x[cc] * N2 + col_y[cc]] = Sz[cc];
    __syncthreads();
    fft_lines<T, true, false>(P, py, nxr, 1, LinesMapped{xrows, N2}, ty);
    fft_lines<T, true, true>(P, px, N2, N2, LinesDirect{1}, tx);
    const double w = wsq ? wsq[b] * wsq[b] : 1.0;
    for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) {
      const double re = P[i].x, im = P[i].y;
      acc[i] += w * (re * re + im * im);
    }
    __syncthreads();
  }
  double* out = part + ((size_t)grp * N3 + z) * N1 * N2;
  for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) out[i] = acc[i] * wfac;
}

// rho[x][y][z] += sum_g part[g][z][x][y]
__global__ void k_density_reduce(int N1, int N2, int N3, int ngrp, const double* __restrict__ part,
                                 double* __restrict__ rho, int accumulate) {
  // consecutive threads take consecutive plane-layout points: the ngrp partial planes are read coalesced
  // (they are most of the traffic); the one C-order write per point is strided
  const int pl = blockIdx.x * blockDim.x + threadIdx.x;
  if (pl >= N1 * N2 * N3) return;
  const int y = pl % N2, x = (pl / N2) % N1, z = pl / (N1 * N2);
  const size_t idx = ((size_t)x * N2 + y) * N3 + z;
  double s = 0.0;
  for (int g = 0; g < ngrp; ++g) s += part[(size_t)g * N1 * N2 * N3 + pl];
  rho[idx] = accumulate ? rho[idx] + s : s;
}

// the same for unscaled FP32 partial planes: rho (+)= wfac sum_g part_g, summed in FP64
__global__ void k_density_reduce32(int N1, int N2, int N3, int ngrp, const float* __restrict__ part, double wfac,
                                   double* __restrict__ rho, int accumulate) {
  const int pl = blockIdx.x * blockDim.x + threadIdx.x;
  if (pl >= N1 * N2 * N3) return;
  const int y = pl % N2, x = (pl / N2) % N1, z = pl / (N1 * N2);
  const size_t idx = ((size_t)x * N2 + y) * N3 + z;
  // the groups summed in a compensated FP32 pair (two-sum; within ~2^-46 of the FP64 sum), converted once
  float hi = 0.f, lo = 0.f;
  for (int g = 0; g < ngrp; ++g) two_sum_acc(hi, lo, part[(size_t)g * N1 * N2 * N3 + pl]);
  const double s = ((double)hi + (double)lo) * wfac;
  rho[idx] = accumulate ? rho[idx] + s : s;
}

template <typename T> static const cplx<T>* twid(const Ctx* c, int ax);
template <> const double2* twid<double>(const Ctx* c, int ax) { return c->d_tw64[ax]; }
template <> const float2* twid<float>(const Ctx* c, int ax) { return c->d_tw32[ax]; }

// rho(r) (+)= wfac sum_b |psi~_b(r)|^2 for nbands orbitals of k-point ik (the FFTs in T, sums in FP64)
template <typename T>
int density_bands(Ctx* c, int ik, int nbands, const cplx<T>* psi, double wfac, double* rho_dev, bool accumulate,
                  const double* wsq) {
  const int N1 = c->N[0], N2 = c->N[1], N3 = c->N[2];
  const int gsize = 8;
  const int ngrp = (nbands + gsize - 1) / gsize;
  if (nbands < 1) return fail(c, PARO_ERR_ARG, "density: no bands");
  double* part = static_cast<double*>(ws_get(c, "dens_part", (size_t)ngrp * c->ngrid * sizeof(double)));
  if (!part) return PARO_ERR_CUDA;
  const size_t smem = (size_t)N1 * N2 * sizeof(double) + (size_t)(N1 + N2 + N1 * N2) * sizeof(cplx<T>);
  const int threads = 512;
  const Basis& B = c->bases[ik];
  cplx<T>* S = static_cast<cplx<T>*>(
      ws_get(c, sizeof(T) == 8 ? "sticks64" : "sticks32", (size_t)nbands * N3 * B.ncol * sizeof(cplx<T>)));
  if (!S) return PARO_ERR_CUDA;
  int st = sticks_inverse<T>(c, ik, nbands, psi, S);
  if (st) return st;
  cudaEvent_t ev = prof_begin(c);
  bool used = false, f32part = false;
  if ((st = density_planes_reg<T>(c, ik, S, nbands, ngrp, gsize, wfac, wsq, part, &used, &f32part))) return st;
  if (!used) {
    if (smem > 227 * 1024) return fail(c, PARO_ERR_ARG, "density: plane too large for shared memory");
    PARO_CU(c, cudaFuncSetAttribute(k_plane_density<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    k_plane_density<T><<<dim3(N3, ngrp), threads, smem, c->stream>>>(
        S, B.ncol, nbands, gsize, B.d_col_x, B.d_col_y, B.d_xrows, B.nxr, c->plan[0], c->plan[1], twid<T>(c, 0),
        twid<T>(c, 1), wfac, wsq, part);
    PARO_LAUNCH(c, "k_plane_density");
  }
  prof_end(c, sizeof(T) == 8 ? "k_plane_density<f64>" : "k_plane_density<f32>", ev);
  if (used && f32part)
    k_density_reduce32<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(N1, N2, N3, ngrp,
                                                                      reinterpret_cast<const float*>(part), wfac,
                                                                      rho_dev, accumulate);
  else
    k_density_reduce<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(N1, N2, N3, ngrp, part, rho_dev, accumulate);
  PARO_LAUNCH(c, "k_density_reduce");
  return PARO_OK;
}

// per-block partial sums of a grid function (fixed chunks, summed on the host in order)
__global__ void k_grid_sum(int n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// a = target / total with total = (Omega/N) sum of the grid partials and target = sum_k w_k fac sum_b
// norms[k][b] (one warp, fixed order); the scale stays on the device
__global__ void k_renorm_scalar(int nblk, const double* __restrict__ part, int nk, int nb, int nrow,
                                const double* __restrict__ wk, double fac, const double* __restrict__ norms,
                                const double* __restrict__ wsq, double dv, double* __restrict__ a) {
  const int lane = threadIdx.x;
  double t = 0.0, g = 0.0;
  for (int i = lane; i < nblk; i += 32) t += part[i];
  for (int k = 0; k < nk; ++k)
    for (int b = lane; b < nrow; b += 32) {
      const size_t o = (size_t)k * nb + b;
      g += wk[k] * fac * (wsq ? wsq[o] * wsq[o] : 1.0) * norms[o];
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    g += __shfl_xor_sync(0xffffffffu, g, o);
  }
  if (lane == 0) *a = (t > 0.0 && g > 0.0) ? g / (t * dv) : 1.0;
}

__global__ void k_grid_scale(int n, const double* __restrict__ a, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= *a;
}

// rho(r) = sum_k w_k sum_b f_kb |psi_kb(r)|^2 / Omega from orbitals in precision T (occupations of the
// context: f = 2 for the lowest nocc bands, or, with smearing, the rows scaled by sqrt(f_kb) first).
// FP32 orbitals: the FP32 transforms' gain (rounded twiddles, FP32 butterflies) biases the density's scale
// by ~1e-7, which the SCF fixed point amplifies; the exact discrete Parseval identity
// (Omega/N) sum_r rho(r) = sum_k w_k sum_b f_kb ||c_kb||^2 restores its normalisation (the norms summed in
// FP64 from the same FP32 rows).
template <typename T>
int density(Ctx* c, const cplx<T>* const* psis, double* rho_dev) {
  if (c->occ.size() != (size_t)c->nk * c->nb) {
    const int st = update_occupations(c);
    if (st) return st;
  }
  const bool renorm = sizeof(T) == 4;
  const int nrow = c->kT > 0 ? c->nocc_eff : c->nocc;
  double* norms = renorm ? static_cast<double*>(ws_get(c, "dens_norms", (size_t)c->nk * c->nb * sizeof(double)))
                         : nullptr;
  if (renorm && !norms) return PARO_ERR_CUDA;
  for (int ik = 0; ik < c->nk; ++ik) {
    int st;
    const int npw = c->bases[ik].npw;
    const cplx<T>* rows = psis[ik];
    // smeared occupations: the density passes weight each band by f (sqrt(f) squared); in the
    // real-wavefunction mode, whose transforms carry two bands, the rows are scaled by sqrt(f) first
    const double* wsq = c->kT > 0 && !gamma_on(c) ? c->d_occ_sqrt + (size_t)ik * c->nb : nullptr;
    if (c->kT > 0 && gamma_on(c)) {
      cplx<T>* y = static_cast<cplx<T>*>(
          ws_get(c, sizeof(T) == 8 ? "dens_scaled64" : "dens_scaled32", (size_t)nrow * npw * sizeof(cplx<T>)));
      if (!y) return PARO_ERR_CUDA;
      if ((st = scale_rows<T>(c, nrow, npw, psis[ik], c->d_occ_sqrt + (size_t)ik * c->nb, y))) return st;
      rows = y;
    }
    const double wfac = (c->kT > 0 ? 1.0 : 2.0) * c->kw[ik] / c->omega;
    int nnorm = nrow;
    if (gamma_on(c)) {  // real orbitals: two per transform, |a + i b|^2 = a^2 + b^2
      st = gamma_density_rows<T>(c, ik, nrow, rows, wfac, rho_dev, ik > 0, &nnorm, &rows);
    } else {
      st = density_bands<T>(c, ik, nrow, rows, wfac, rho_dev, ik > 0, wsq);
    }
    if (st) return st;
    if (renorm) {
      if ((st = band_norms<T>(c, nnorm, npw, rows, npw, norms + (size_t)ik * c->nb))) return st;
      if (nnorm < nrow)  // packed rows: ||a + i b||^2 = ||a||^2 + ||b||^2; the slots behind them count zero
        PARO_CU(c, cudaMemsetAsync(norms + (size_t)ik * c->nb + nnorm, 0, (size_t)(nrow - nnorm) * sizeof(double),
                                   c->stream));
    }
  }
  if (!renorm) return PARO_OK;
  const int nblk = 304;
  double* part = static_cast<double*>(ws_get(c, "dens_sum_part", (nblk + 1) * sizeof(double)));
  double* wk = static_cast<double*>(ws_get(c, "dens_kw", (size_t)c->nk * sizeof(double)));
  if (!part || !wk) return PARO_ERR_CUDA;
  if (int st = h2d_async(c, "dens_kw", wk, c->kw.data(), c->nk * sizeof(double))) return st;
  k_grid_sum<<<nblk, 256, 0, c->stream>>>(c->ngrid, rho_dev, part);
  PARO_LAUNCH(c, "k_grid_sum");
  // smeared: each norm weighted by f (the scaled rows of the real-wavefunction mode already carry it);
  // otherwise f = 2
  const bool weighted = c->kT > 0 && !gamma_on(c);
  k_renorm_scalar<<<1, 32, 0, c->stream>>>(nblk, part, c->nk, c->nb, nrow, wk, c->kT > 0 ? 1.0 : 2.0, norms,
                                           weighted ? c->d_occ_sqrt : nullptr, c->omega / c->ngrid, part + nblk);
  PARO_LAUNCH(c, "k_renorm_scalar");
  k_grid_scale<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, part + nblk, rho_dev);
  PARO_LAUNCH(c, "k_grid_scale");
  return PARO_OK;
}

template int density_bands<double>(Ctx*, int, int, const double2*, double, double*, bool, const double*);
template int density_bands<float>(Ctx*, int, int, const float2*, double, double*, bool, const double*);
template int density<double>(Ctx*, const double2* const*, double*);
template int density<float>(Ctx*, const float2* const*, double*);

// ------------------------------------------------------------------------------------------------
// energy terms
// ------------------------------------------------------------------------------------------------
// per block partial sums of w_b * sum_g kin_g |c_bg|^2 over blocks (band, chunk)
// FP32 orbitals (mixed precision): FP32 terms summed in an FP32 two-sum pair, no FP64 per coefficient
// (grid: band x chunk of the row; part[b * gridDim.y + chunk])
template <typename T>
__global__ void k_kinetic(int npw, const cplx<T>* __restrict__ psi, const T* __restrict__ kin, double* part) {
  __shared__ double red[32];
  const int b = blockIdx.x, len = (npw + gridDim.y - 1) / gridDim.y;
  const int g0 = blockIdx.y * len, g1 = min(npw, g0 + len);
  double s = 0.0;
  if (sizeof(T) == 4) {
    float hi = 0.f, lo = 0.f;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      const cplx<T> v = psi[(size_t)b * npw + g];
      two_sum_acc(hi, lo, (float)(kin[g] * (v.x * v.x + v.y * v.y)));
    }
    s = (double)hi + (double)lo;
  } else {
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      const cplx<T> v = psi[(size_t)b * npw + g];
      s += (double)kin[g] * ((double)v.x * v.x + (double)v.y * v.y);
    }
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.y + blockIdx.y] = s;
}

// sum_p D_p |P[p][b]|^2 per band b
__global__ void k_nonlocal(int nproj, int nb, const double2* __restrict__ P, const double* __restrict__ dvec,
                           double* part) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int p = threadIdx.x; p < nproj; p += blockDim.x) {
    const double2 v = P[(size_t)p * nb + b];
    s += dvec[p] * (v.x * v.x + v.y * v.y);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[b] = s;
}

// per block partials of sum V_loc rho and sum rho eps_xc(rho)
template <typename R>
__global__ void k_grid_energies(int n, const double* __restrict__ vloc, const double* __restrict__ rho,
                                double* __restrict__ part) {
  __shared__ double red[32];
  double sl = 0.0, sx = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double e;
    if constexpr (sizeof(R) == 8) {
      e = lda_pz_eps64(rho[i]);
    } else {
      R ef, vf;
      lda_pz<R>((R)rho[i], &ef, &vf);
      e = (double)ef;
    }
    sl += vloc[i] * rho[i];
    sx += rho[i] * e;
  }
  sl = block_sum(sl, red);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = sl;
  sx = block_sum(sx, red);
  if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = sx;
}

int energy_terms(Ctx* c, const double* rho_dev, double terms[7]) {
  for (int i = 0; i < 7; ++i) terms[i] = 0.0;
  // every partial sum lands in one buffer, read back with a single synchronisation:
  // [kinetic: nk x nocc x kKch][nonlocal: nk x nocc][V_loc rho, rho eps_xc: 2 x 304][Hartree blocks]
  constexpr int kKch = 4;  // chunks of each row for the kinetic sums (enough CTAs to fill the GPU)
  if (c->occ.size() != (size_t)c->nk * c->nb) {
    const int st = update_occupations(c);
    if (st) return st;
  }
  const int nocc = c->kT > 0 ? c->nocc_eff : c->nocc;  // bands with an occupation
  const int nblk = 304, nh = hartree_blocks(c), nkb = c->nk * nocc, nkk = nkb * kKch;
  const size_t ntot = (size_t)nkk + nkb + 2 * nblk + nh;
  double* part = static_cast<double*>(ws_get(c, "energy_part", ntot * sizeof(double)));
  double2* z = static_cast<double2*>(ws_get(c, "grid_c0", (size_t)c->ngrid * sizeof(double2)));
  if (!part || !z) return PARO_ERR_CUDA;
  double *pk = part, *pn = part + nkk, *pg = pn + nkb, *ph = pg + 2 * nblk;
  int st;
  for (int ik = 0; ik < c->nk; ++ik) {
    const Basis& B = c->bases[ik];
    const dim3 gk(nocc, kKch);
    if (c->prec == PARO_MIXED && B.d_psi32)
      k_kinetic<float><<<gk, 256, 0, c->stream>>>(B.npw, B.d_psi32, B.d_kin32, pk + (size_t)ik * nocc * kKch);
    else
      k_kinetic<double><<<gk, 256, 0, c->stream>>>(B.npw, B.d_psi, B.d_kin, pk + (size_t)ik * nocc * kKch);
    PARO_LAUNCH(c, "k_kinetic");
    if (c->have_kb) {
      double2* P = static_cast<double2*>(ws_get(c, "kb_proj", (size_t)c->nproj * c->nb * sizeof(double2)));
      if (!P) return PARO_ERR_CUDA;
      // <beta|psi>: FP64 on the FP64 path; the mixed path projects its FP32 orbitals in FP32 with the
      // sums carried in a two-sum pair (the energy sum itself stays FP64)
      st = c->prec == PARO_MIXED && B.d_psi32
               ? gemm_cn<float, float, float>(c, c->nproj, nocc, B.npw, B.d_beta32, B.npw, B.d_psi32, B.npw, P,
                                              nocc, false, true)
               : gemm_cn<double, double, double>(c, c->nproj, nocc, B.npw, B.d_beta, B.npw, B.d_psi, B.npw, P,
                                                 nocc, false);
      if (st) return st;
      k_nonlocal<<<nocc, 256, 0, c->stream>>>(c->nproj, nocc, P, c->d_dvec, pn + (size_t)ik * nocc);
      PARO_LAUNCH(c, "k_nonlocal");
    }
  }
  // eps_xc per point in FP64 on both paths (an FP32 evaluation shifts E_xc of the 64-atom cell by ~1e-5 Ha;
  // one pass over the grid, a few tens of microseconds in FP64)
  k_grid_energies<double><<<nblk, 256, 0, c->stream>>>(c->ngrid, c->d_vloc, rho_dev, pg);
  PARO_LAUNCH(c, "k_grid_energies");
  if ((st = hartree_g(c, rho_dev, z, ph, false))) return st;
  std::vector<double> h(ntot);
  PARO_CU(c, cudaMemcpyAsync(h.data(), part, ntot * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  for (int ik = 0; ik < c->nk; ++ik) {
    double sk = 0, sn = 0;
    for (int b = 0; b < nocc; ++b) {
      const double f = c->occ[(size_t)ik * c->nb + b];
      double kb = 0;
      for (int ch = 0; ch < kKch; ++ch) kb += h[((size_t)ik * nocc + b) * kKch + ch];
      sk += f * kb;
      sn += f * h[nkk + (size_t)ik * nocc + b];
    }
    terms[PARO_E_KINETIC] += c->kw[ik] * sk;
    if (c->have_kb) terms[PARO_E_NONLOCAL] += c->kw[ik] * sn;
  }
  double sl = 0, sx = 0, sh = 0;
  for (int i = 0; i < nblk; ++i) {
    sl += h[nkk + nkb + 2 * i];
    sx += h[nkk + nkb + 2 * i + 1];
  }
  for (int i = 0; i < nh; ++i) sh += h[nkk + nkb + 2 * nblk + i];
  const double dv = c->omega / c->ngrid;
  terms[PARO_E_LOCAL] = dv * sl;
  terms[PARO_E_XC] = dv * sx;
  terms[PARO_E_HARTREE] = hartree_energy(c, sh);
  terms[PARO_E_EWALD] = c->e_ewald;
  // with smearing the total is the Mermin free energy E - T S
  terms[PARO_E_TOTAL] = terms[0] + terms[1] + terms[2] + terms[3] + terms[4] + terms[5] + (c->kT > 0 ? c->mts : 0.0);
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Pulay (DIIS) mixing: rho_new = sum_i a_i (rho_in^i + beta R^i), a minimising ||sum a_i R^i|| with
// sum a_i = 1 over the stored history (a ring buffer of depth <= pulay_cap).
// ------------------------------------------------------------------------------------------------
__global__ void k_pulay_push(int n, const double* __restrict__ rin, const double* __restrict__ rout,
                             double* __restrict__ hr, double* __restrict__ hres) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  hr[i] = rin[i];
  hres[i] = rout[i] - rin[i];
}

// part[blk][i*m + j] = block partial of <R_i, R_j> (i <= j)
// <res_new, res_slot[i]> for the m slots of the history (the new residual is one of them): one pass over
// the vectors, per-CTA partials part[block * 16 + i]. The other pairs were formed when the later of the
// two arrived and are kept in the Gram cache.
__global__ void __launch_bounds__(256) k_pulay_dots(int n, int m, const double* __restrict__ hres,
                                                    const int* __restrict__ slot, int snew,
                                                    double* __restrict__ part) {
  __shared__ double red[32];
  double acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0;
  const double* rn = hres + (size_t)snew * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const double x = rn[t];
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < m) acc[i] = fma(x, hres[(size_t)slot[i] * n + t], acc[i]);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (i >= m) break;
    const double v = block_sum(acc[i], red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 16 + i] = v;
    __syncthreads();
  }
}

// one CTA: the new row of the Gram cache from the partials, then the bordered system
//   [G 1; 1^T 0] [a; lambda] = [0; 1]
// by Gauss-Jordan elimination with partial pivoting, every step spread over the CTA's threads
__global__ void __launch_bounds__(256) k_pulay_solve(int m, int nblk, const double* __restrict__ part,
                                                     const int* __restrict__ slot, int snew,
                                                     double* __restrict__ gram, double* __restrict__ coef) {
  __shared__ double a[17][19];
  __shared__ double fac[17];
  __shared__ int s_piv;
  {  // the block partials of each new dot summed by one warp (lane-strided, then a shuffle tree)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < m; i += nw) {
      double s = 0.0;
      for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * 16 + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        gram[snew * 16 + slot[i]] = s;
        gram[slot[i] * 16 + snew] = s;
      }
    }
  }
  __syncthreads();
  const int n = m + 1;  // unknowns; column n holds the right-hand side
  for (int ij = threadIdx.x; ij < n * (n + 1); ij += blockDim.x) {
    const int i = ij / (n + 1), j = ij - i * (n + 1);
    double v;
    if (j == n) v = i == m ? 1.0 : 0.0;
    else if (i < m && j < m) v = gram[slot[i] * 16 + slot[j]];
    else v = i == j ? 0.0 : 1.0;  // the border of ones, zero in the corner
    a[i][j] = v;
  }
  __syncthreads();
  for (int col = 0; col < n; ++col) {
    if (threadIdx.x < 32) {  // pivot: the largest |a[r][col]| for r >= col, the first one on ties
      const int r = col + (int)threadIdx.x;
      double best = r < n ? fabs(a[r][col]) : -1.0;
      int at = r < n ? r : n;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, at, o);
        if (ob > best || (ob == best && oa < at)) {
          best = ob;
          at = oa;
        }
      }
      if (threadIdx.x == 0) s_piv = at;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != col)
      for (int k = threadIdx.x; k <= n; k += blockDim.x) {
        const double t = a[col][k];
        a[col][k] = a[piv][k];
        a[piv][k] = t;
      }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) fac[r] = r == col ? 0.0 : a[r][col] / a[col][col];
    __syncthreads();
    for (int ij = threadIdx.x; ij < n * (n + 1 - col); ij += blockDim.x) {
      const int r = ij / (n + 1 - col), k = col + ij - r * (n + 1 - col);
      if (r != col) a[r][k] -= fac[r] * a[col][k];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) coef[i] = a[i][n] / a[i][i];
}

__global__ void k_pulay_mix(int n, int m, const double* __restrict__ hr, const double* __restrict__ hres,
                            const int* __restrict__ slot, const double* __restrict__ coef, double beta,
                            double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = 0.0;
  for (int i = 0; i < m; ++i) {
    const size_t o = (size_t)slot[i] * n + t;
    s += coef[i] * (hr[o] + beta * hres[o]);
  }
  out[t] = s;
}

int pulay_mix(Ctx* c, const double* rho_out, int depth, double beta) {
  if (depth < 1 || depth > 16) return fail(c, PARO_ERR_ARG, "pulay depth must be in [1, 16]");
  const int n = c->ngrid;
  if (!c->d_pulay_rho || c->pulay_cap != depth) {
    if (c->d_pulay_rho) { cudaFree(c->d_pulay_rho); cudaFree(c->d_pulay_res); }
    PARO_CU(c, cudaMalloc(&c->d_pulay_rho, (size_t)depth * n * sizeof(double)));
    PARO_CU(c, cudaMalloc(&c->d_pulay_res, (size_t)depth * n * sizeof(double)));
    if (!c->d_pulay_gram) PARO_CU(c, cudaMalloc(&c->d_pulay_gram, 16 * 16 * sizeof(double)));
    c->pulay_cap = depth;
    c->pulay_n = 0;
    c->pulay_head = 0;
  }
  const int slot_new = c->pulay_head;
  k_pulay_push<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->d_rho_in, rho_out, c->d_pulay_rho + (size_t)slot_new * n,
                                                       c->d_pulay_res + (size_t)slot_new * n);
  PARO_LAUNCH(c, "k_pulay_push");
  c->pulay_head = (c->pulay_head + 1) % depth;
  if (c->pulay_n < depth) ++c->pulay_n;
  const int m = c->pulay_n;
  // oldest first
  c->pulay_slots.resize(m);
  for (int i = 0; i < m; ++i) c->pulay_slots[i] = ((c->pulay_head - m + i) % depth + depth) % depth;
  int* dslot = static_cast<int*>(ws_get(c, "pulay_slot", 16 * sizeof(int)));
  const int nblk = 152;
  double* part = static_cast<double*>(ws_get(c, "pulay_part", (size_t)nblk * 16 * sizeof(double)));
  double* coef = static_cast<double*>(ws_get(c, "pulay_coef", 16 * sizeof(double)));
  if (!dslot || !part || !coef) return PARO_ERR_CUDA;
  if (int st = h2d_async(c, "pulay_slots", dslot, c->pulay_slots.data(), m * sizeof(int))) return st;
  k_pulay_dots<<<nblk, 256, 0, c->stream>>>(n, m, c->d_pulay_res, dslot, slot_new, part);
  PARO_LAUNCH(c, "k_pulay_dots");
  k_pulay_solve<<<1, 256, 0, c->stream>>>(m, nblk, part, dslot, slot_new, c->d_pulay_gram, coef);
  PARO_LAUNCH(c, "k_pulay_solve");
  k_pulay_mix<<<(n + 255) / 256, 256, 0, c->stream>>>(n, m, c->d_pulay_rho, c->d_pulay_res, dslot, coef, beta,
                                                      c->d_rho_in);
  PARO_LAUNCH(c, "k_pulay_mix");
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// Ewald energy of point ions Z in a neutralising background (host, FP64)
// ------------------------------------------------------------------------------------------------
double ewald(const Ctx* c) {
  const double* L = c->lat;
  const double omega = c->omega;
  const double Z = c->Z;
  const int nat = c->nat;
  const double eta = std::sqrt(kPi) / std::cbrt(omega);
  const double tol = 1e-16;
  double rcut = 1.0;
  while (std::erfc(eta * rcut) / rcut > tol) rcut *= 1.2;
  int nmax[3];
  for (int i = 0; i < 3; ++i) {
    const double* u = L + 3 * ((i + 1) % 3);
    const double* v = L + 3 * ((i + 2) % 3);
    const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    const double h = omega / std::sqrt(cx * cx + cy * cy + cz * cz);  // layer spacing
    nmax[i] = (int)std::ceil(rcut / h) + 1;
  }
  double ereal = 0;
  for (int i = 0; i < nat; ++i)
    for (int j = 0; j < nat; ++j)
      for (int a = -nmax[0]; a <= nmax[0]; ++a)
        for (int b = -nmax[1]; b <= nmax[1]; ++b)
          for (int cc = -nmax[2]; cc <= nmax[2]; ++cc) {
            double d[3];
            for (int x = 0; x < 3; ++x)
              d[x] = c->pos[i * 3 + x] - c->pos[j * 3 + x] + a * L[x] + b * L[3 + x] + cc * L[6 + x];
            const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r > 1e-12 && r < rcut) ereal += 0.5 * Z * Z * std::erfc(eta * r) / r;
          }
  const double gcut = 2.0 * eta * std::sqrt(-std::log(tol));
  int gm[3];
  for (int i = 0; i < 3; ++i) {
    const double len = std::sqrt(L[3 * i] * L[3 * i] + L[3 * i + 1] * L[3 * i + 1] + L[3 * i + 2] * L[3 * i + 2]);
    gm[i] = (int)std::ceil(gcut * len / (2 * kPi)) + 1;
  }
  double erec = 0;
  for (int a = -gm[0]; a <= gm[0]; ++a)
    for (int b = -gm[1]; b <= gm[1]; ++b)
      for (int cc = -gm[2]; cc <= gm[2]; ++cc) {
        double g[3];
        for (int x = 0; x < 3; ++x) g[x] = a * c->bmat[x] + b * c->bmat[3 + x] + cc * c->bmat[6 + x];
        const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        if (g2 <= 0 || g2 >= gcut * gcut) continue;
        double sr = 0, si = 0;
        for (int I = 0; I < nat; ++I) {
          const double ph = g[0] * c->pos[I * 3] + g[1] * c->pos[I * 3 + 1] + g[2] * c->pos[I * 3 + 2];
          sr += Z * std::cos(ph);
          si += Z * std::sin(ph);
        }
        erec += (sr * sr + si * si) * std::exp(-g2 / (4 * eta * eta)) / g2;
      }
  erec *= 2 * kPi / omega;
  const double eself = -eta / std::sqrt(kPi) * nat * Z * Z;
  const double ebg = -kPi * (nat * Z) * (nat * Z) / (2 * omega * eta * eta);
  return ereal + erec + eself + ebg;
}

}  // namespace paro
