// libparo C ABI (include/paro.h): context setup and the ParO / SCF drivers that sequence the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/paro.h"
#include "paro_ctx.h"

struct paro_ctx {
  paro::Ctx c;
};

namespace paro {

static thread_local std::string g_create_err;
static const double kPi = 3.14159265358979323846;

Ctx* unwrap(paro_ctx* h) { return h ? &h->c : nullptr; }

int fail(Ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  return fail(c, PARO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* ws_get(Ctx* c, const char* name, size_t bytes) {
  auto it = c->ws.find(name);
  if (it != c->ws.end() && it->second.second >= bytes) return it->second.first;
  if (it != c->ws.end()) {
    cudaStreamSynchronize(c->stream);
    cudaFree(it->second.first);
    c->ws.erase(it);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    cuda_fail(c, e, "workspace allocation");
    return nullptr;
  }
  c->ws[name] = std::make_pair(p, bytes);
  return p;
}

// pinned buffer `name` of at least `bytes`, once its previous copy has completed
static Ctx::Pinned* pinned_get(Ctx* c, const char* name, size_t bytes) {
  Ctx::Pinned& p = c->pinned[name];
  if (p.ev && cudaEventSynchronize(p.ev) != cudaSuccess) return nullptr;
  if (p.bytes < bytes) {
    if (p.h) cudaFreeHost(p.h);
    p.h = nullptr;
    p.bytes = 0;
    if (cudaMallocHost(&p.h, bytes) != cudaSuccess) return nullptr;
    p.bytes = bytes;
  }
  if (!p.ev && cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return &p;
}

int h2d_async(Ctx* c, const char* name, void* dst, const void* src, size_t bytes) {
  if (!bytes) return PARO_OK;
  Ctx::Pinned* p = pinned_get(c, name, bytes);
  if (!p) return fail(c, PARO_ERR_CUDA, std::string("pinned staging buffer ") + name);
  std::memcpy(p->h, src, bytes);
  PARO_CU(c, cudaMemcpyAsync(dst, p->h, bytes, cudaMemcpyHostToDevice, c->stream));
  PARO_CU(c, cudaEventRecord(p->ev, c->stream));
  return PARO_OK;
}

int d2h_async(Ctx* c, const char* name, const void* src, size_t bytes, void** h) {
  Ctx::Pinned* p = pinned_get(c, name, bytes > 0 ? bytes : 8);
  if (!p) return fail(c, PARO_ERR_CUDA, std::string("pinned read-back buffer ") + name);
  if (bytes) PARO_CU(c, cudaMemcpyAsync(p->h, src, bytes, cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaEventRecord(p->ev, c->stream));
  if (h) *h = p->h;
  return PARO_OK;
}

int pinned_wait(Ctx* c, const char* name) {
  auto it = c->pinned.find(name);
  if (it == c->pinned.end() || !it->second.ev) return PARO_OK;
  PARO_CU(c, cudaEventSynchronize(it->second.ev));
  return PARO_OK;
}

// ------------------------------------------------------------------------------------------------
// setup helpers
// ------------------------------------------------------------------------------------------------
static int smooth23_above(int m) {
  for (int x = m + 1;; ++x) {
    int y = x;
    while (y % 2 == 0) y /= 2;
    while (y % 3 == 0) y /= 3;
    if (y == 1) return x;
  }
}

static FftPlan make_plan(int n) {
  FftPlan p;
  p.n = n;
  p.nst = 0;
  int e2 = 0, e3 = 0, y = n;
  while (y % 2 == 0) { y /= 2; ++e2; }
  while (y % 3 == 0) { y /= 3; ++e3; }
  int n8 = e2 / 3, rem = e2 % 3;
  std::vector<int> r;
  if (rem == 1 && n8 > 0) { --n8; r.push_back(4); r.push_back(4); rem = 0; }
  for (int i = 0; i < n8; ++i) r.insert(r.begin(), 8);
  if (rem == 2) r.push_back(4);
  if (rem == 1) r.push_back(2);
  for (int i = 0; i < e3; ++i) r.push_back(3);
  for (size_t i = 0; i < r.size() && i < 8; ++i) p.rad[p.nst++] = r[i];
  return p;
}

FftPlan fft_plan(int n) { return make_plan(n); }

// Miller indices with |k+G|^2/2 <= ecut, lexicographic (n1, n2, n3); kinetic energies.
static void sphere(const Ctx* c, const double kf[3], double ecut, std::vector<int>& mil, std::vector<double>& kin) {
  const double* B = c->bmat;
  double kc[3];
  for (int x = 0; x < 3; ++x) kc[x] = kf[0] * B[x] + kf[1] * B[3 + x] + kf[2] * B[6 + x];
  const double gmax = std::sqrt(2.0 * ecut);
  int lim[3];
  for (int i = 0; i < 3; ++i) {
    const double* a = c->lat + 3 * i;
    const double len = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    lim[i] = (int)std::floor(gmax * len / (2 * kPi) + std::fabs(kf[i])) + 1;
  }
  mil.clear();
  kin.clear();
  for (int n1 = -lim[0]; n1 <= lim[0]; ++n1)
    for (int n2 = -lim[1]; n2 <= lim[1]; ++n2)
      for (int n3 = -lim[2]; n3 <= lim[2]; ++n3) {
        double q[3];
        for (int x = 0; x < 3; ++x) q[x] = kc[x] + (n1 * B[x] + n2 * B[3 + x] + n3 * B[6 + x]);
        const double e = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (e <= ecut) {
          mil.push_back(n1);
          mil.push_back(n2);
          mil.push_back(n3);
          kin.push_back(e);
        }
      }
}

template <typename T>
static int upload(Ctx* c, T** d, const std::vector<T>& h) {
  PARO_CU(c, cudaMalloc(d, std::max<size_t>(h.size(), 1) * sizeof(T)));
  if (!h.empty()) PARO_CU(c, cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PARO_OK;
}

static int build_basis(Ctx* c, Basis& b) {
  std::vector<int>& mil = b.miller;
  sphere(c, b.kfrac, c->ecut, mil, b.kin);
  b.npw = (int)b.kin.size();
  std::vector<int> col_x, col_y, col_off, g_col(b.npw), g_z(b.npw);
  for (int g = 0; g < b.npw; ++g) {
    const int n1 = mil[3 * g], n2 = mil[3 * g + 1], n3 = mil[3 * g + 2];
    if (g == 0 || n1 != mil[3 * (g - 1)] || n2 != mil[3 * (g - 1) + 1]) {
      col_x.push_back(((n1 % c->N[0]) + c->N[0]) % c->N[0]);
      col_y.push_back(((n2 % c->N[1]) + c->N[1]) % c->N[1]);
      col_off.push_back(g);
    }
    g_col[g] = (int)col_x.size() - 1;
    g_z[g] = ((n3 % c->N[2]) + c->N[2]) % c->N[2];
  }
  b.ncol = (int)col_x.size();
  col_off.push_back(b.npw);
  std::vector<int> xr(col_x);
  std::sort(xr.begin(), xr.end());
  xr.erase(std::unique(xr.begin(), xr.end()), xr.end());
  b.nxr = (int)xr.size();
  std::vector<int> xrc(c->N[0], -1);
  for (int r = 0; r < b.nxr; ++r) xrc[xr[r]] = r;
  std::vector<int> stick_of((size_t)b.nxr * c->N[1], -1);
  for (int cc = 0; cc < b.ncol; ++cc) stick_of[(size_t)xrc[col_x[cc]] * c->N[1] + col_y[cc]] = cc;
  std::vector<float> kin32(b.kin.begin(), b.kin.end());
  int st;
  if ((st = upload(c, &b.d_miller, mil)) || (st = upload(c, &b.d_kin, b.kin)) || (st = upload(c, &b.d_kin32, kin32)) ||
      (st = upload(c, &b.d_col_x, col_x)) || (st = upload(c, &b.d_col_y, col_y)) ||
      (st = upload(c, &b.d_col_off, col_off)) || (st = upload(c, &b.d_g_col, g_col)) ||
      (st = upload(c, &b.d_g_z, g_z)) || (st = upload(c, &b.d_xrows, xr)) || (st = upload(c, &b.d_xrow_c, xrc)) ||
      (st = upload(c, &b.d_stick_of, stick_of)))
    return st;
  return PARO_OK;
}

// Every device array of a basis (plane-wave tables, KB projectors, orbitals); the host tables are kept.
static void free_basis(Basis& b) {
  void** ps[] = {(void**)&b.d_miller, (void**)&b.d_kin,    (void**)&b.d_kin32,  (void**)&b.d_col_x,
                 (void**)&b.d_col_y,  (void**)&b.d_col_off, (void**)&b.d_g_col,  (void**)&b.d_g_z,
                 (void**)&b.d_xrows,  (void**)&b.d_xrow_c, (void**)&b.d_stick_of, (void**)&b.d_beta,   (void**)&b.d_beta32, (void**)&b.d_beta_img_cn, (void**)&b.d_beta_img_wx, (void**)&b.d_prec_base,
                 (void**)&b.d_mg,
                 (void**)&b.d_psi,    (void**)&b.d_hpsi,   (void**)&b.d_psi32,  (void**)&b.d_hpsi32};
  for (void** p : ps) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

// The plane-wave basis of every k-point for the cutoff c->ecut (Eq. e3) and the FFT grid of the alias-free
// rule, N_i = smallest 2^a 3^b above m_V,i + s_psi,i (m_V: largest |n_i| of the density sphere
// |G|^2/2 <= 4 E_cut; s_psi: span of n_i over every k's basis), with the grid's twiddle tables. Earlier
// bases (their orbitals included) and twiddles are freed; k-points (kfrac, kcart) are kept.
static int setup_bases(Ctx* c) {
  const double ecut = c->ecut;
  int span[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
  {
    std::vector<int> mil;
    std::vector<double> kin;
    const double zero[3] = {0, 0, 0};
    sphere(c, zero, 4.0 * ecut, mil, kin);
    for (size_t g = 0; g < kin.size(); ++g)
      for (int i = 0; i < 3; ++i) mv[i] = std::max(mv[i], std::abs(mil[3 * g + i]));
  }
  for (int ik = 0; ik < c->nk; ++ik) {
    std::vector<int> mil;
    std::vector<double> kin;
    sphere(c, c->bases[ik].kfrac, ecut, mil, kin);
    if ((int)kin.size() < c->nb) return fail(c, PARO_ERR_ARG, "fewer plane waves than bands");
    for (int i = 0; i < 3; ++i) {
      int lo = 1 << 30, hi = -(1 << 30);
      for (size_t g = 0; g < kin.size(); ++g) {
        lo = std::min(lo, mil[3 * g + i]);
        hi = std::max(hi, mil[3 * g + i]);
      }
      span[i] = std::max(span[i], hi - lo);
    }
  }
  for (int i = 0; i < 3; ++i) {
    c->N[i] = smooth23_above(mv[i] + span[i]);
    c->plan[i] = make_plan(c->N[i]);
  }
  c->ngrid = c->N[0] * c->N[1] * c->N[2];
  c->max_npw = 0;
  for (int ik = 0; ik < c->nk; ++ik) {
    Basis& b = c->bases[ik];
    free_basis(b);
    b.have_psi = false;
    b.hx_recur = 0;
    b.eps.clear();
    b.res.clear();
    int st = build_basis(c, b);
    if (st) return st;
    c->max_npw = std::max(c->max_npw, b.npw);
  }
  for (int ax = 0; ax < 3; ++ax) {
    if (c->d_tw64[ax]) cudaFree(c->d_tw64[ax]);
    if (c->d_tw32[ax]) cudaFree(c->d_tw32[ax]);
    c->d_tw64[ax] = nullptr;
    c->d_tw32[ax] = nullptr;
  }
  int st = build_twiddles(c);
  if (st) return st;
  return check_fft_support(c, c->prec == PARO_MIXED ? 8 : 16);
}

// PCG shift per k-point: below the spectrum of H by the bound V_min + sum of the negative KB terms, - 1/2
static void update_sigma(Ctx* c) {
  c->sigma_k.assign(c->nk, 0.0);
  for (int ik = 0; ik < c->nk; ++ik) {
    double lb = c->vmin;
    if (c->have_kb)
      for (int I = 0; I < c->nat; ++I) {
        const double* m = &c->beta_norm2_max[((size_t)ik * c->nat + I) * 2];
        if (c->D[2 * I] < 0) lb += c->D[2 * I] * m[0];
        if (c->D[2 * I + 1] < 0) lb += c->D[2 * I + 1] * 3.0 * m[1];
      }
    c->sigma_k[ik] = lb - 0.5;
  }
}

int veff_stats(Ctx* c) {
  if (c->vstats_pending) {
    int st = pinned_wait(c, "vstats");
    if (st) return st;
    const double* h = static_cast<const double*>(c->pinned["vstats"].h);
    c->vmean = h[0] / c->ngrid;
    c->vmin = h[1];
    c->vstats_pending = false;
  }
  update_sigma(c);
  return PARO_OK;
}

// The mixed-precision iteration works on the FP32 orbitals and H psi; their FP64 copies are formed only
// when a call reads them (orbitals out, Algorithm 2's right-hand sides, a restart, a cutoff step, a batch).
int fp64_current(Ctx* c, Basis& b) {
  const size_t n = (size_t)c->nb * b.npw;
  if (b.psi64_stale) {
    if (int st = convert<float, double>(c, n, b.d_psi32, b.d_psi)) return st;
    b.psi64_stale = false;
  }
  if (b.hpsi64_stale) {
    if (int st = convert<float, double>(c, n, b.d_hpsi32, b.d_hpsi)) return st;
    b.hpsi64_stale = false;
  }
  return PARO_OK;
}

static int alloc_orbitals(Ctx* c, Basis& b) {
  if (!b.d_psi) {
    PARO_CU(c, cudaMalloc(&b.d_psi, (size_t)c->nb * b.npw * sizeof(double2)));
    PARO_CU(c, cudaMalloc(&b.d_hpsi, (size_t)c->nb * b.npw * sizeof(double2)));
  }
  if (c->prec == PARO_MIXED && !b.d_psi32) {
    PARO_CU(c, cudaMalloc(&b.d_psi32, (size_t)c->nb * b.npw * sizeof(float2)));
    PARO_CU(c, cudaMalloc(&b.d_hpsi32, (size_t)c->nb * b.npw * sizeof(float2)));
  }
  return PARO_OK;
}

__global__ void k_hermitize(int n, double2* __restrict__ a) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  if (i < j) return;
  const double2 lo = a[(size_t)i * n + j], up = a[(size_t)j * n + i];
  const double2 h = make_double2(0.5 * (lo.x + up.x), 0.5 * (lo.y - up.y));
  a[(size_t)i * n + j] = h;
  a[(size_t)j * n + i] = make_double2(h.x, -h.y);
}

// Orbitals in the working precision: FP64 path d_psi / d_hpsi, mixed path d_psi32 / d_hpsi32.
template <typename T> static cplx<T>* psi_of(Basis& b);
template <> double2* psi_of<double>(Basis& b) { return b.d_psi; }
template <> float2* psi_of<float>(Basis& b) { return b.d_psi32; }
template <typename T> static cplx<T>* hpsi_of(Basis& b);
template <> double2* hpsi_of<double>(Basis& b) { return b.d_hpsi; }
template <> float2* hpsi_of<float>(Basis& b) { return b.d_hpsi32; }

static const char* wsn(bool f64, const char* a, const char* b) { return f64 ? a : b; }

// Rayleigh-Ritz in the span of the nx rows of X (Algorithm 1 step 4): Cholesky-orthonormalise
// (Y = conj(L)^{-1} X, skipped when X is already orthonormal), H_sub = Y^H H Y, H_sub C = C diag(eps),
// psi = first nb rows of C^T Y, H psi = C^T (H Y), residual norms. T = double: every step in FP64.
// T = float (mixed): the Cholesky apply, H Y and the rotations in FP32; the Gram and H_sub products
// accumulated in FP64 (upper halves, mirrored); Cholesky, eigensolver and residual norms in FP64.
// HX (may be null): H X of the rows of X at the potential of the inner solves; dvplane (may be null): the
// change of the local potential since then (V-plane layout). With HX, H Y = G H X (+ dV Y) replaces the
// H application.
// defer: the residual norms and the tensor-core flag are left to project_readback (the SCF iteration
// reads them after its energy)
template <typename T>
static int project(Ctx* c, int ik, cplx<T>* X, int nx, bool orthonormal, cplx<T>* HX, const T* dvplane,
                   bool defer = false);
static int project_readback(Ctx* c, int ik);
template <typename T>
static int project(Ctx* c, int ik, cplx<T>* X, int nx, bool orthonormal) {
  return project<T>(c, ik, X, nx, orthonormal, nullptr, nullptr);
}
template <typename T>
static int project(Ctx* c, int ik, cplx<T>* X, int nx, bool orthonormal, cplx<T>* HX, const T* dvplane, bool defer) {
  Basis& b = c->bases[ik];
  const int npw = b.npw, nb = c->nb;
  const bool f64 = sizeof(T) == 8;
  double2* S = static_cast<double2*>(ws_get(c, "proj_S", (size_t)nx * nx * sizeof(double2)));
  double2* G = static_cast<double2*>(ws_get(c, "proj_G", (size_t)nx * nx * sizeof(double2)));
  cplx<T>* Y = static_cast<cplx<T>*>(ws_get(c, wsn(f64, "proj_Y64", "proj_Y32"), (size_t)nx * npw * sizeof(cplx<T>)));
  cplx<T>* HY =
      static_cast<cplx<T>*>(ws_get(c, wsn(f64, "proj_HY64", "proj_HY32"), (size_t)nx * npw * sizeof(cplx<T>)));
  double* w = static_cast<double*>(ws_get(c, "proj_w", (size_t)nx * sizeof(double)));
  double* res = static_cast<double*>(ws_get(c, "proj_res", (size_t)nx * sizeof(double)));
  if (!S || !G || !Y || !HY || !w || !res) return PARO_ERR_CUDA;
  int st;
  if (orthonormal) {
    Y = X;
  } else {
    {
      ProfTag t(c, "gram");
      if ((st = gemm_cn<T, T, T>(c, nx, nx, npw, X, npw, X, npw, S, nx, true, true))) return st;
      if (gamma_on(c) && (st = gamma_real_matrix(c, nx, S))) return st;  // real orbitals: real Gram
      if ((st = chol_inv(c, nx, S, G))) return st;
    }
    ProfTag t(c, "orth");
    if ((st = gemm_wx<T, T>(c, nx, npw, nx, G, nx, true, nullptr, X, npw, Y, npw, 0.0, nullptr, true))) return st;
    if (HX && (st = gemm_wx<T, T>(c, nx, npw, nx, G, nx, true, nullptr, HX, npw, HY, npw, 0.0, nullptr, true)))
      return st;
  }
  {
    ProfTag t(c, "rr");
    bool done = false;
    if (HX) {
      if (orthonormal)
        PARO_CU(c, cudaMemcpyAsync(HY, HX, (size_t)nx * npw * sizeof(cplx<T>), cudaMemcpyDeviceToDevice,
                                   c->stream));
      done = true;
      if (dvplane && (st = apply_dv<T>(c, ik, nx, Y, HY, dvplane, &done))) return st;
    }
    if (!done && (st = apply_h<T>(c, ik, nx, Y, HY, 0.0, nullptr))) return st;
  }
  const int* hinfo = nullptr;
  const float* hemax = nullptr;
  {
    ProfTag t(c, "hsub");
    if ((st = gemm_cn<T, T, T>(c, nx, nx, npw, Y, npw, HY, npw, S, nx, true, true))) return st;
    if (gamma_on(c) && (st = gamma_real_matrix(c, nx, S))) return st;  // real orbitals: real symmetric H_sub
    k_hermitize<<<(nx * nx + 255) / 256, 256, 0, c->stream>>>(nx, S);
    PARO_LAUNCH(c, "k_hermitize");
    // mixed: one refinement step (FP64 Ritz values, vectors well below the FP32 level of the orbitals); its
    // cluster check is read back below, with the Ritz values
    if ((st = f64 ? eigh(c, nx, S, w, G) : eigh_mixed(c, nx, S, w, G, 1, true, &hinfo, &hemax))) return st;  // G <- C
  }
  // the rotations, H psi of the new orbitals and their residual norms
  auto rotate = [&]() -> int {
    ProfTag t(c, "rot");
    int s2;
    if ((s2 = gemm_wx<T, T>(c, nb, npw, nx, G, nx, false, nullptr, Y, npw, psi_of<T>(b), npw, 0.0))) return s2;
    if ((s2 = gemm_wx<T, T>(c, nb, npw, nx, G, nx, false, nullptr, HY, npw, hpsi_of<T>(b), npw, 0.0))) return s2;
    if (gamma_on(c)) {  // real orbitals stay real (the rotation's rounding may not keep c(-G) = conj c(G))
      if ((s2 = gamma_real_rows<T>(c, ik, nb, psi_of<T>(b))) || (s2 = gamma_real_rows<T>(c, ik, nb, hpsi_of<T>(b))))
        return s2;
    }
    if (!f64) {
      b.psi64_stale = b.hpsi64_stale = true;
      return residual_norms32(c, nb, npw, b.d_psi32, b.d_hpsi32, w, res);
    }
    return residual_norms(c, nb, npw, b.d_psi, b.d_hpsi, w, res);
  };
  // The Ritz values come back while the rotations run: the host waits only for the eigensolve, and the
  // caller's next work (occupations, energy) is queued behind the rotations. Residual norms and the
  // tensor-core flag are read by project_readback.
  const std::string rname = "proj_res_" + std::to_string(ik);
  void *he = nullptr, *hr = nullptr;
  const int* htc = nullptr;
  auto finish = [&]() -> int {
    int s2;
    if ((s2 = d2h_async(c, "proj_eps", w, nb * sizeof(double), &he)) || (s2 = rotate()) ||
        (s2 = d2h_async(c, rname.c_str(), res, nb * sizeof(double), &hr)) || (s2 = tc_flag_readback(c, &htc)) ||
        (s2 = pinned_wait(c, "proj_eps")))
      return s2;
    return PARO_OK;
  };
  if ((st = finish())) return st;
  if (hemax && (st = pinned_wait(c, "eig_warm_emax"))) return st;
  if (hemax && !eigh_mixed_accept(c, *hemax)) {
    // a warm start that went on without waiting and was not accepted (rare near convergence): the FP32
    // solve, then the rotations again from the unchanged Rayleigh-Ritz basis
    hinfo = nullptr;
    if ((st = eigh_mixed(c, nx, S, w, G, 1, false, &hinfo)) || (st = finish())) return st;
  }
  if (hinfo && (*hinfo & (1 | 4 | 8))) {
    // a cluster the mixed refinement could not resolve (rare): the FP64 solver, then the rotations again
    // from the unchanged Rayleigh-Ritz basis
    if ((st = eigh_mixed_check(c, nx, S, w, G, *hinfo)) || (st = finish())) return st;
  }
  b.eps.assign(static_cast<const double*>(he), static_cast<const double*>(he) + nb);
  b.res_pending = true;
  b.have_psi = true;
  return defer ? PARO_OK : project_readback(c, ik);
}

// The residual norms of the last Rayleigh-Ritz step of k-point ik and the tensor-core error flag.
static int project_readback(Ctx* c, int ik) {
  Basis& b = c->bases[ik];
  if (!b.res_pending) return PARO_OK;
  const std::string rname = "proj_res_" + std::to_string(ik);
  int st = pinned_wait(c, rname.c_str());
  if (st) return st;
  const double* hr = static_cast<const double*>(c->pinned[rname].h);
  b.res.assign(hr, hr + c->nb);
  b.res_pending = false;
  auto it = c->pinned.find("tc_err");
  if (it != c->pinned.end() && it->second.h) {
    if ((st = pinned_wait(c, "tc_err"))) return st;
    if (*static_cast<const int*>(it->second.h)) return fail(c, PARO_ERR_TIMEOUT, "tensor-core product: mbarrier wait gave up");
  }
  return PARO_OK;
}

template <typename T>
__global__ void k_axpy_rows(int npw, cplx<T>* __restrict__ y, const cplx<T>* __restrict__ x, T sx) {
  const int b = blockIdx.y;
  const size_t o = (size_t)b * npw;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x)
    y[o + g] = cadd(y[o + g], cscale(x[o + g], sx));
}

// rhs_b = -(H psi_b - eps_b psi_b) (Algorithms 2 and 3's correction equations), formed in FP64 from the
// current orbitals and stored in T
template <typename T>
static int source_rhs(Ctx* c, int ik, cplx<T>* rhs) {
  Basis& b = c->bases[ik];
  const int nb = c->nb, npw = b.npw;
  double* f = static_cast<double*>(ws_get(c, "rhs_f", (size_t)nb * sizeof(double)));
  double2* tmp = static_cast<double2*>(ws_get(c, "rhs_tmp", (size_t)nb * npw * sizeof(double2)));
  if (!f || !tmp) return PARO_ERR_CUDA;
  int st;
  if ((st = fp64_current(c, b)) || (st = h2d_async(c, "rhs_f", f, b.eps.data(), nb * sizeof(double)))) return st;
  if ((st = scale_rows<double>(c, nb, npw, b.d_psi, f, tmp))) return st;
  k_axpy_rows<double><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, tmp, b.d_hpsi, -1.0);
  PARO_LAUNCH(c, "k_axpy_rows");
  if (sizeof(T) == 8) {
    PARO_CU(c, cudaMemcpyAsync(rhs, tmp, (size_t)nb * npw * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    return PARO_OK;
  }
  return convert<double, float>(c, (size_t)nb * npw, tmp, reinterpret_cast<float2*>(rhs));
}

// Source problems of all bands of k-point ik; solutions in x (T), started at psi (Algorithm 1) or 0.
template <typename T>
static int solve_sources(Ctx* c, int ik, bool alg2, double rel_tol, int max_it, cplx<T>* x, cplx<T>* hx = nullptr) {
  Basis& b = c->bases[ik];
  const int nb = c->nb, npw = b.npw;
  const bool f64 = sizeof(T) == 8;
  int st;
  if (!alg2) {
    // Algorithm 1: rhs = (eps - sigma) psi, started at the orbitals, whose H psi the last Rayleigh-Ritz step
    // left in hpsi; the solver's first pass forms rhs, the start vectors and their residuals together
    double* f = static_cast<double*>(ws_get(c, "rhs_f", (size_t)nb * sizeof(double)));
    if (!f) return PARO_ERR_CUDA;
    if ((st = veff_stats(c))) return st;
    std::vector<double> hf(nb);
    for (int i = 0; i < nb; ++i) hf[i] = b.eps[i] - c->sigma_k[ik];
    if ((st = h2d_async(c, "rhs_f", f, hf.data(), nb * sizeof(double)))) return st;
    return pcg_run<T>(c, ik, nb, nullptr, x, false, rel_tol, max_it, nullptr, hpsi_of<T>(b), hx, psi_of<T>(b), f);
  }
  cplx<T>* rhs = static_cast<cplx<T>*>(ws_get(c, wsn(f64, "src_rhs64", "src_rhs32"), (size_t)nb * npw * sizeof(cplx<T>)));
  if (!rhs) return PARO_ERR_CUDA;
  if ((st = source_rhs<T>(c, ik, rhs))) return st;
  return pcg_run<T>(c, ik, nb, rhs, x, true, rel_tol, max_it, nullptr, nullptr, nullptr);
}

template <typename T>
__global__ void k_compact_rows(int npw, int nb, cplx<T>* __restrict__ dst, const cplx<T>* __restrict__ src,
                               const int* __restrict__ map) {
  const int r = blockIdx.y;
  const int from = map[r];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x)
    dst[(size_t)(nb + r) * npw + g] = src[(size_t)from * npw + g];
}

// Algorithm 2: rows [psi, e] of X with e projected out of span{psi}; corrections whose remaining
// norm is at most 1e-10 are left out (they add nothing to the span).
template <typename T>
static int build_alg2_basis(Ctx* c, int ik, cplx<T>* E, cplx<T>* X, int* nx_out) {
  Basis& b = c->bases[ik];
  const int nb = c->nb, npw = b.npw;
  const bool f64 = sizeof(T) == 8;
  double2* P = static_cast<double2*>(ws_get(c, "alg2_P", (size_t)nb * nb * sizeof(double2)));
  double* nrm = static_cast<double*>(ws_get(c, "alg2_nrm", (size_t)nb * sizeof(double)));
  int* map = static_cast<int*>(ws_get(c, "alg2_map", (size_t)nb * sizeof(int)));
  cplx<T>* tmp = static_cast<cplx<T>*>(ws_get(c, wsn(f64, "alg2_tmp64", "alg2_tmp32"), (size_t)nb * npw * sizeof(cplx<T>)));
  if (!P || !nrm || !map || !tmp) return PARO_ERR_CUDA;
  cplx<T>* psi = psi_of<T>(b);
  int st;
  // P[i][j] = <psi_i, e_j>;  e_j -= sum_i psi_i P[i][j]
  if ((st = gemm_cn<T, T, T>(c, nb, nb, npw, psi, npw, E, npw, P, nb, false, true))) return st;
  if (gamma_on(c) && (st = gamma_real_matrix(c, nb, P))) return st;
  if ((st = gemm_wx<T, T>(c, nb, npw, nb, P, nb, false, nullptr, psi, npw, tmp, npw, 0.0))) return st;
  k_axpy_rows<T><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, E, tmp, (T)-1);
  PARO_LAUNCH(c, "k_axpy_rows");
  if ((st = band_norms<T>(c, nb, npw, E, npw, nrm))) return st;
  std::vector<double> h(nb);
  PARO_CU(c, cudaMemcpyAsync(h.data(), nrm, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  std::vector<int> keep;
  for (int i = 0; i < nb; ++i)
    if (std::sqrt(h[i]) > 1e-10) keep.push_back(i);
  PARO_CU(c, cudaMemcpyAsync(X, psi, (size_t)nb * npw * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, c->stream));
  if (!keep.empty()) {
    PARO_CU(c, cudaMemcpyAsync(map, keep.data(), keep.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    k_compact_rows<T><<<dim3((npw + 255) / 256, (int)keep.size()), 256, 0, c->stream>>>(npw, nb, X, E, map);
    PARO_LAUNCH(c, "k_compact_rows");
  }
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  *nx_out = nb + (int)keep.size();
  return PARO_OK;
}

static cudaEvent_t prof_event(Ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

cudaEvent_t prof_begin(Ctx* c) {
  if (!c->prof) return nullptr;
  cudaEvent_t a = prof_event(c);
  if (a) cudaEventRecord(a, c->stream);
  return a;
}

void prof_end(Ctx* c, const char* name, cudaEvent_t a) {
  if (!c->prof || !a) return;
  cudaEvent_t b = prof_event(c);
  if (!b) {
    c->prof_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, c->stream);
  c->prof_ev.push_back({c->prof_tag ? std::string(c->prof_tag) + ":" + name : std::string(name), a, b});
}

// Occupations of the current Ritz values. kT = 0: f = 2 for the lowest nocc bands of every k-point.
// kT > 0 (Fermi-Dirac): mu by bisection on the electron count sum_k w_k sum_i f_ik = 2 nocc, and
// -T S = -kT sum_k w_k sum_i 2 s(g), s(g) = -(g ln g + (1 - g) ln(1 - g)), g = f/2.
static double fermi_g(double x) {  // 1 / (1 + e^x) without overflow
  return x > 0 ? std::exp(-x) / (1.0 + std::exp(-x)) : 1.0 / (1.0 + std::exp(x));
}

int update_occupations(Ctx* c) {
  const int nk = c->nk, nb = c->nb;
  // unchanged Ritz values, kT and electron count leave the occupations as they are (the SCF iteration asks
  // at its start for those of the values its last energy evaluation used)
  std::vector<double> key{c->kT, (double)c->nocc};
  if (c->kT > 0) {
    key.reserve(2 + (size_t)nk * nb);
    for (int ik = 0; ik < nk; ++ik) {
      if ((int)c->bases[ik].eps.size() < nb) return fail(c, PARO_ERR_STATE, "occupations: no Ritz values");
      key.insert(key.end(), c->bases[ik].eps.begin(), c->bases[ik].eps.begin() + nb);
    }
  }
  if (key == c->occ_key && c->occ.size() == (size_t)nk * nb) return PARO_OK;
  c->occ_key.clear();
  c->occ.assign((size_t)nk * nb, 0.0);
  if (c->kT <= 0) {
    for (int ik = 0; ik < nk; ++ik)
      for (int i = 0; i < c->nocc; ++i) c->occ[(size_t)ik * nb + i] = 2.0;
    c->nocc_eff = c->nocc;
    c->mu = 0;
    c->mts = 0;
    c->occ_key.swap(key);
    return PARO_OK;
  }
  double lo = 1e300, hi = -1e300;
  for (int ik = 0; ik < nk; ++ik)
    for (int i = 0; i < nb; ++i) {
      lo = std::min(lo, c->bases[ik].eps[i]);
      hi = std::max(hi, c->bases[ik].eps[i]);
    }
  const double kT = c->kT, nel = 2.0 * c->nocc;
  lo -= 40 * kT + 1;  // N(lo) < nel < N(hi)
  hi += 40 * kT + 1;
  // N(mu) - nel and its derivative sum_k w_k sum_i 2 g (1 - g) / kT
  auto excess = [&](double mu, double* dn) {
    double n = 0, d = 0;
    for (int ik = 0; ik < nk; ++ik)
      for (int i = 0; i < nb; ++i) {
        const double g = fermi_g((c->bases[ik].eps[i] - mu) / kT);
        n += c->kw[ik] * 2.0 * g;
        d += c->kw[ik] * 2.0 * g * (1.0 - g);
      }
    *dn = d / kT;
    return n - nel;
  };
  // N(mu) = nel by Newton's method inside a shrinking bracket, bisecting whenever the Newton point leaves the
  // bracket or the step has not at least halved since the one before; ends when mu no longer moves
  double mu = 0.5 * (lo + hi), d = 0, step = hi - lo, step_prev = step;
  double f = excess(mu, &d);
  for (int it = 0; it < 400 && f != 0.0; ++it) {
    if (f < 0) lo = mu;
    else hi = mu;
    const double newton = d > 0 ? mu - f / d : lo;
    const bool take = newton > lo && newton < hi && std::fabs(2.0 * f) <= std::fabs(step_prev * d);
    const double next = take ? newton : 0.5 * (lo + hi);
    step_prev = step;
    step = next - mu;
    if (next == mu || next <= lo || next >= hi) break;
    mu = next;
    f = excess(mu, &d);
  }
  c->mu = mu;
  double ts = 0;
  int neff = 0;
  std::vector<double> sq((size_t)nk * nb);
  for (int ik = 0; ik < nk; ++ik)
    for (int i = 0; i < nb; ++i) {
      const double g = fermi_g((c->bases[ik].eps[i] - c->mu) / kT);
      const size_t o = (size_t)ik * nb + i;
      c->occ[o] = 2.0 * g;
      sq[o] = std::sqrt(2.0 * g);
      if (g > 0) ts -= c->kw[ik] * 2.0 * kT * g * std::log(g);
      if (g < 1) ts -= c->kw[ik] * 2.0 * kT * (1.0 - g) * std::log1p(-g);
      if (2.0 * g > 1e-15) neff = std::max(neff, i + 1);
    }
  c->mts = -ts;
  c->nocc_eff = std::max(neff, 1);
  if (!c->d_occ_sqrt) PARO_CU(c, cudaMalloc(&c->d_occ_sqrt, (size_t)nk * nb * sizeof(double)));
  int st = h2d_async(c, "occ_sqrt", c->d_occ_sqrt, sq.data(), sq.size() * sizeof(double));
  if (st) return st;
  c->occ_key.swap(key);
  return PARO_OK;
}

static double max_occ_resid(const Ctx* c) {
  double m = 0;
  for (const Basis& b : c->bases)
    for (int i = 0; i < c->nocc && i < (int)b.res.size(); ++i) m = std::max(m, b.res[i]);
  return m;
}

// step 3 of Algorithm 1/2 for k-point ik: the new basis rows in X (T), count in nx
// HX (may be null; Algorithm 1 only): receives H X of the sources, carried through the inner solves.
template <typename T>
static int source_step(Ctx* c, int ik, int alg, double rel_tol, int max_it, cplx<T>* X, int* nx,
                       cplx<T>* HX = nullptr);
template <typename T>
static int source_step(Ctx* c, int ik, int alg, double rel_tol, int max_it, cplx<T>* X, int* nx, cplx<T>* HX) {
  const bool alg2 = alg == PARO_ALG2 || alg == PARO_ALG3;
  const int npw = c->bases[ik].npw;
  cplx<T>* E = X;
  if (alg2) {
    E = static_cast<cplx<T>*>(ws_get(c, wsn(sizeof(T) == 8, "alg2_E64", "alg2_E32"), (size_t)c->nb * npw * sizeof(cplx<T>)));
    if (!E) return PARO_ERR_CUDA;
  }
  // Algorithm 3: the projected correction equations with lambda_i = eps_i, by batched MINRES
  Basis& b = c->bases[ik];
  int st = alg == PARO_ALG3
               ? minres_run<T>(c, ik, c->nb, psi_of<T>(b), hpsi_of<T>(b), b.eps.data(), E, rel_tol, max_it, nullptr)
               : solve_sources<T>(c, ik, alg2, rel_tol, max_it, E, alg2 ? nullptr : HX);
  if (st) return st;
  if (!alg2) {
    *nx = c->nb;
    return PARO_OK;
  }
  return build_alg2_basis<T>(c, ik, E, X, nx);
}

// ||S - I||_F up to which the mixed SCF iteration orthonormalises its sources by the first-order factor:
// the rows are then orthonormal to 3 tol^2 = 7.5e-9, below the FP32 rounding of the rows themselves.
static const double kOrthFirstTol = 5e-5;

// Cholesky-orthonormalise the first nx rows of X in place (Y = conj(L)^{-1} X); Gram in FP64.
template <typename T>
static int orthonormalize(Ctx* c, int ik, cplx<T>* X, int nx, cplx<T>* HX = nullptr, bool defer = false) {
  const int npw = c->bases[ik].npw;
  const bool f64 = sizeof(T) == 8;
  double2* S = static_cast<double2*>(ws_get(c, "proj_S", (size_t)nx * nx * sizeof(double2)));
  double2* G = static_cast<double2*>(ws_get(c, "proj_G", (size_t)nx * nx * sizeof(double2)));
  cplx<T>* Y = static_cast<cplx<T>*>(ws_get(c, wsn(f64, "proj_Y64", "proj_Y32"), (size_t)nx * npw * sizeof(cplx<T>)));
  if (!S || !G || !Y) return PARO_ERR_CUDA;
  int st;
  {
    ProfTag t(c, "gram");
    if ((st = gemm_cn<T, T, T>(c, nx, nx, npw, X, npw, X, npw, S, nx, true, true))) return st;
    if (gamma_on(c) && (st = gamma_real_matrix(c, nx, S))) return st;
    // mixed-precision SCF iteration: near convergence the sources are orthonormal to ~1e-5 and the
    // first-order factor (orthonormal to ~3 ||E||^2, below the FP32 rounding of the rows) replaces the
    // FP64 Cholesky, decided on the device; the Cholesky kernel then returns at once
    int* skip = nullptr;
    bool cl_ok = false;
    if (defer && !f64 && (st = chol_cluster_available(c, nx, &cl_ok))) return st;
    if (cl_ok && (st = orth_first_order(c, nx, S, G, kOrthFirstTol, &skip))) return st;
    if ((st = chol_inv(c, nx, S, G, defer, skip))) return st;
  }
  ProfTag t(c, "orth");
  if ((st = gemm_wx<T, T>(c, nx, npw, nx, G, nx, true, nullptr, X, npw, Y, npw, 0.0, nullptr, true))) return st;
  PARO_CU(c, cudaMemcpyAsync(X, Y, (size_t)nx * npw * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, c->stream));
  if (HX) {  // H Y = G (H X): the same combination of the known H X
    if ((st = gemm_wx<T, T>(c, nx, npw, nx, G, nx, true, nullptr, HX, npw, Y, npw, 0.0, nullptr, true))) return st;
    PARO_CU(c, cudaMemcpyAsync(HX, Y, (size_t)nx * npw * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, c->stream));
  }
  return PARO_OK;
}

// Workspace for 2 n_bands rows of k-point ik in T
template <typename T>
static cplx<T>* rows_ws(Ctx* c, const char* base, int ik) {
  std::string name = std::string(base) + (sizeof(T) == 8 ? "64_" : "32_") + std::to_string(ik);
  return static_cast<cplx<T>*>(ws_get(c, name.c_str(), (size_t)2 * c->nb * c->bases[ik].npw * sizeof(cplx<T>)));
}

// Takes the FP64 orbitals in d_psi with the eigenvalue estimates in b.eps as the current state (no
// orthonormalisation, no Rayleigh-Ritz): the working-precision copy, H psi under the current potential
// and the residual norms.
static int adopt_orbitals(Ctx* c, int ik) {
  Basis& b = c->bases[ik];
  int st;
  double* w = static_cast<double*>(ws_get(c, "state_eps", (size_t)c->nb * sizeof(double)));
  double* res = static_cast<double*>(ws_get(c, "state_res", (size_t)c->nb * sizeof(double)));
  if (!w || !res) return PARO_ERR_CUDA;
  PARO_CU(c, cudaMemcpyAsync(w, b.eps.data(), c->nb * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  b.psi64_stale = false;  // the FP64 orbitals are the ones given
  if (c->prec == PARO_MIXED) {
    if ((st = convert<double, float>(c, (size_t)c->nb * b.npw, b.d_psi, b.d_psi32))) return st;
    if ((st = apply_h<float>(c, ik, c->nb, b.d_psi32, b.d_hpsi32, 0.0, nullptr))) return st;
    b.hpsi64_stale = true;
    if ((st = residual_norms32(c, c->nb, b.npw, b.d_psi32, b.d_hpsi32, w, res))) return st;
  } else {
    b.hpsi64_stale = false;
    if ((st = apply_h<double>(c, ik, c->nb, b.d_psi, b.d_hpsi, 0.0, nullptr)) ||
        (st = residual_norms(c, c->nb, b.npw, b.d_psi, b.d_hpsi, w, res)))
      return st;
  }
  b.res.resize(c->nb);
  PARO_CU(c, cudaMemcpyAsync(b.res.data(), res, c->nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  b.hx_recur = 0;
  b.have_psi = true;
  return PARO_OK;
}

// Rayleigh-Ritz of the span of the current orbitals (after a change of potential or a restart)
static int reproject(Ctx* c, int ik) {
  Basis& b = c->bases[ik];
  const size_t n = (size_t)c->nb * b.npw;
  if (c->prec == PARO_MIXED) {
    float2* X = rows_ws<float>(c, "X", ik);
    if (!X) return PARO_ERR_CUDA;
    int st = fp64_current(c, b);
    if (st) return st;
    st = convert<double, float>(c, n, b.d_psi, X);
    return st ? st : project<float>(c, ik, X, c->nb, false);
  }
  double2* X = rows_ws<double>(c, "X", ik);
  if (!X) return PARO_ERR_CUDA;
  PARO_CU(c, cudaMemcpyAsync(X, b.d_psi, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  return project<double>(c, ik, X, c->nb, false);
}

// Algorithm 1 forms H of the Rayleigh-Ritz basis from the inner solves' own products (H X carried
// through the iteration, G H X after orthonormalisation, plus dV Y when the potential moved). After
// kHxRefresh such iterations one applies H directly, so the FP32 rounding of the carried H psi cannot
// accumulate over many iterations.
static const int kHxRefresh = 8;
static bool carry_hx(Basis& b, int alg) {
  const bool carry = alg == PARO_ALG1 && b.hx_recur < kHxRefresh;
  b.hx_recur = carry ? b.hx_recur + 1 : 0;
  return carry;
}

// One ParO step (Algorithm 1 or 2) of k-point ik at the current potential.
template <typename T>
static int paro_step_k(Ctx* c, int ik, int alg, double rel_tol, int max_it) {
  cplx<T>* X = rows_ws<T>(c, "X", ik);
  if (!X) return PARO_ERR_CUDA;
  cplx<T>* HX = carry_hx(c->bases[ik], alg) ? rows_ws<T>(c, "HX", ik) : nullptr;
  int nx = c->nb;
  int st = source_step<T>(c, ik, alg, rel_tol, max_it, X, &nx, HX);
  return st ? st : project<T>(c, ik, X, nx, false, HX, nullptr);
}

template <typename T> static T* vplane_dev(Ctx* c);
template <> double* vplane_dev<double>(Ctx* c) { return c->d_vplane; }
template <> float* vplane_dev<float>(Ctx* c) { return c->d_vplane32; }

// dv = v_new - dv (in place: dv holds the old planes on entry)
template <typename T>
__global__ void k_plane_delta(int n, const T* __restrict__ vnew, T* __restrict__ dv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dv[i] = vnew[i] - dv[i];
}

// The merged SCF iteration in precision T (see paro_scf_step).
template <typename T>
static int scf_iteration(Ctx* c, const paro_scf_opts* o) {
  std::vector<cplx<T>*> xs(c->nk), hxs(c->nk, nullptr);
  std::vector<int> nxs(c->nk);
  int st;
  c->chol_pending.clear();  // flags left by an iteration that stopped early
  // the source solutions x_i carry the occupations of the eps_i^n they are solved with
  if ((st = update_occupations(c))) return st;
  bool carry = false;  // some k-point carries H X this iteration (then dV is needed)
  for (int ik = 0; ik < c->nk; ++ik) {
    xs[ik] = rows_ws<T>(c, "X", ik);
    if (!xs[ik]) return PARO_ERR_CUDA;
    if (carry_hx(c->bases[ik], o->alg)) {
      if (!(hxs[ik] = rows_ws<T>(c, "HX", ik))) return PARO_ERR_CUDA;
      carry = true;
    }
    if ((st = source_step<T>(c, ik, o->alg, o->inner_rel_tol, o->inner_max_it, xs[ik], &nxs[ik], hxs[ik])))
      return st;
    // a Cholesky breakdown is reported below, before anything of the state changes
    if ((st = orthonormalize<T>(c, ik, xs[ik], nxs[ik], hxs[ik], true))) return st;
  }
  // the potential planes of the inner solves, to form dV once the mixing has moved the potential
  T* dv = nullptr;
  if (carry) {
    dv = static_cast<T*>(ws_get(c, sizeof(T) == 8 ? "dv_plane64" : "dv_plane32", (size_t)c->ngrid * sizeof(T)));
    if (!dv) return PARO_ERR_CUDA;
    PARO_CU(c, cudaMemcpyAsync(dv, vplane_dev<T>(c), (size_t)c->ngrid * sizeof(T), cudaMemcpyDeviceToDevice,
                               c->stream));
  }
  // rho_in^{n+1/2} = Pulay(rho_in^n, rho[X]) (Algorithm 2: rho of the previous orbitals)
  double* rho_out = static_cast<double*>(ws_get(c, "scf_rho_out", (size_t)c->ngrid * sizeof(double)));
  if (!rho_out) return PARO_ERR_CUDA;
  std::vector<const cplx<T>*> dens_src(c->nk);
  for (int ik = 0; ik < c->nk; ++ik) dens_src[ik] = o->alg == PARO_ALG1 ? xs[ik] : psi_of<T>(c->bases[ik]);  // 2, 3
  {
    ProfTag t(c, "mix");
    if ((st = density<T>(c, dens_src.data(), rho_out))) return st;
    if ((st = chol_check(c))) return st;  // the GPU still has the density pass queued
    if ((st = pulay_mix(c, rho_out, o->pulay_depth, o->pulay_beta))) return st;
    if ((st = veff_from_density(c, c->d_rho_in, nullptr, nullptr))) return st;
  }
  if (carry) {
    k_plane_delta<T><<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, vplane_dev<T>(c), dv);
    PARO_LAUNCH(c, "k_plane_delta");
  }
  // step 4: Rayleigh-Ritz with V(rho_in^{n+1/2}) in the already orthonormal span
  for (int ik = 0; ik < c->nk; ++ik)
    if ((st = project<T>(c, ik, xs[ik], nxs[ik], true, hxs[ik], dv, true))) return st;
  return PARO_OK;
}

// density of the current orbitals, in the working precision
static int current_density(Ctx* c, double* rho) {
  int st = update_occupations(c);
  if (st) return st;
  if (c->prec == PARO_MIXED) {
    std::vector<const float2*> ps(c->nk);
    for (int ik = 0; ik < c->nk; ++ik) ps[ik] = c->bases[ik].d_psi32;
    return density<float>(c, ps.data(), rho);
  }
  std::vector<const double2*> ps(c->nk);
  for (int ik = 0; ik < c->nk; ++ik) ps[ik] = c->bases[ik].d_psi;
  return density<double>(c, ps.data(), rho);
}

}  // namespace paro

using namespace paro;

// y += a x on the grid
__global__ void k_axpy_grid(int n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void k_real_part_api(int n, const double2* __restrict__ z, double* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = z[i].x;
}

// ------------------------------------------------------------------------------------------------
// Cutoff ladder (Algorithm 1 step 2): orbitals embedded in the larger basis, grid functions carried to
// the new grid by Fourier interpolation
// ------------------------------------------------------------------------------------------------
// z = v - vl (vl may be null)
__global__ void k_rest_complex(int n, const double* __restrict__ v, const double* __restrict__ vl,
                               double2* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = make_double2(v[i] - (vl ? vl[i] : 0.0), 0.0);
}

// fnew[n mod Nnew] = scale * fold[n mod Nold] for every signed index n with 2 |n_i| < Nold_i (the old
// grid's Nyquist planes are dropped); fnew is zero elsewhere (cleared by the caller)
__global__ void k_fourier_carry(int o1, int o2, int o3, int m1, int m2, int m3, const double2* __restrict__ fold,
                                double2* __restrict__ fnew, double scale) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= o1 * o2 * o3) return;
  const int j3 = idx % o3, j2 = (idx / o3) % o2, j1 = idx / (o2 * o3);
  const int n1 = j1 * 2 < o1 ? j1 : j1 - o1, n2 = j2 * 2 < o2 ? j2 : j2 - o2, n3 = j3 * 2 < o3 ? j3 : j3 - o3;
  if (2 * abs(n1) >= o1 || 2 * abs(n2) >= o2 || 2 * abs(n3) >= o3) return;
  const int k1 = (n1 + m1) % m1, k2 = (n2 + m2) % m2, k3 = (n3 + m3) % m3;
  const double2 v = fold[idx];
  fnew[((size_t)k1 * m2 + k2) * m3 + k3] = make_double2(v.x * scale, v.y * scale);
}

// row b of the larger basis: dst[b][map[g]] = src[b][g] (the other coefficients were cleared)
__global__ void k_prolong(int npw_old, int npw_new, const int* __restrict__ map, const double2* __restrict__ src,
                          double2* __restrict__ dst) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw_old; g += gridDim.x * blockDim.x)
    dst[(size_t)b * npw_new + map[g]] = src[(size_t)b * npw_old + g];
}

static int set_ecut(Ctx* c, double ecut_new) {
  int st;
  const int o[3] = {c->N[0], c->N[1], c->N[2]};
  const int ngold = c->ngrid;
  // 1. the carried grid function's Fourier coefficients on the old grid: the SCF input density, or the
  //    rest V_eff - V_loc of a set potential
  const bool carry_rho = c->have_rho && c->d_rho_in;
  const bool carry_rest = !carry_rho && c->have_veff;
  double2* fold = nullptr;
  if (carry_rho || carry_rest) {
    PARO_CU(c, cudaMalloc(&fold, (size_t)ngold * sizeof(double2)));
    k_rest_complex<<<(ngold + 255) / 256, 256, 0, c->stream>>>(ngold, carry_rho ? c->d_rho_in : c->d_veff,
                                                              carry_rest && c->have_pp ? c->d_vloc : nullptr, fold);
    PARO_LAUNCH(c, "k_rest_complex");
    if ((st = fft3d<double>(c, fold, false))) return st;
  }
  // 2. the old level's orbitals (FP64), Miller lists and eigenvalue estimates
  std::vector<double2*> old_psi(c->nk, nullptr);
  std::vector<std::vector<int>> old_mil(c->nk);
  std::vector<std::vector<double>> old_eps(c->nk);
  std::vector<int> old_npw(c->nk);
  for (int ik = 0; ik < c->nk; ++ik) {
    Basis& b = c->bases[ik];
    if (!b.have_psi) continue;
    if ((st = fp64_current(c, b))) return st;
    old_psi[ik] = b.d_psi;
    b.d_psi = nullptr;
    old_mil[ik] = b.miller;
    old_eps[ik] = b.eps;
    old_npw[ik] = b.npw;
  }
  // 3. everything sized by the grid or the basis is rebuilt
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  for (auto& kv : c->ws) cudaFree(kv.second.first);
  c->ws.clear();
  double** grid_bufs[] = {&c->d_vloc, &c->d_veff, &c->d_vplane, &c->d_rho_in, &c->d_pulay_rho, &c->d_pulay_res};
  for (double** p : grid_bufs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (c->d_vplane32) cudaFree(c->d_vplane32);
  c->d_vplane32 = nullptr;
  c->pulay_n = c->pulay_head = 0;
  c->have_inv_g2 = false;
  c->have_tw_half = false;
  c->have_veff = false;
  c->ecut = ecut_new;
  c->scf_iter = c->scf_small = 0;
  if ((st = setup_bases(c))) return st;
  if (c->gamma_real && (st = gamma_build_table(c, 0))) return st;
  if (c->have_pp && (st = build_vloc(c))) return st;
  if (c->have_kb && (st = build_beta(c))) return st;
  // 4. the carried function on the new grid: f(j') = sum_n F(n) exp(2 pi i n.j'/N'), F = fold / N_old
  if (fold) {
    double2* fnew = static_cast<double2*>(ws_get(c, "grid_c0", (size_t)c->ngrid * sizeof(double2)));
    double* fr = static_cast<double*>(ws_get(c, "grid_r1", (size_t)c->ngrid * sizeof(double)));
    if (!fnew || !fr) return PARO_ERR_CUDA;
    PARO_CU(c, cudaMemsetAsync(fnew, 0, (size_t)c->ngrid * sizeof(double2), c->stream));
    k_fourier_carry<<<(ngold + 255) / 256, 256, 0, c->stream>>>(o[0], o[1], o[2], c->N[0], c->N[1], c->N[2], fold,
                                                               fnew, 1.0 / ngold);
    PARO_LAUNCH(c, "k_fourier_carry");
    if ((st = fft3d<double>(c, fnew, true))) return st;
    k_real_part_api<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, fnew, fr);
    PARO_LAUNCH(c, "k_real_part");
    PARO_CU(c, cudaStreamSynchronize(c->stream));
    cudaFree(fold);
    if (carry_rho) {
      PARO_CU(c, cudaMalloc(&c->d_rho_in, (size_t)c->ngrid * sizeof(double)));
      PARO_CU(c, cudaMemcpyAsync(c->d_rho_in, fr, (size_t)c->ngrid * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
      if ((st = veff_from_density(c, c->d_rho_in, nullptr, nullptr))) return st;
    } else {
      if (c->have_pp) {
        k_axpy_grid<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, 1.0, c->d_vloc, fr);
        PARO_LAUNCH(c, "k_axpy_grid");
      }
      if ((st = set_veff_device(c, fr))) return st;
    }
    }
  // 5. the orbitals embedded in the new bases, eigenvalue estimates kept
  for (int ik = 0; ik < c->nk; ++ik) {
    if (!old_psi[ik]) continue;
    Basis& b = c->bases[ik];
    std::map<long long, int> where;
    auto key = [](int a, int bb, int cc) { return ((long long)(a + 4096) * 8192 + (bb + 4096)) * 8192 + (cc + 4096); };
    for (int g = 0; g < b.npw; ++g) where[key(b.miller[3 * g], b.miller[3 * g + 1], b.miller[3 * g + 2])] = g;
    std::vector<int> map(old_npw[ik]);
    for (int g = 0; g < old_npw[ik]; ++g) {
      auto it = where.find(key(old_mil[ik][3 * g], old_mil[ik][3 * g + 1], old_mil[ik][3 * g + 2]));
      if (it == where.end()) return fail(c, PARO_ERR_STATE, "paro_set_ecut: old basis not inside the new one");
      map[g] = it->second;
    }
    int* dmap = static_cast<int*>(ws_get(c, "prolong_map", (size_t)old_npw[ik] * sizeof(int)));
    if (!dmap) return PARO_ERR_CUDA;
    if ((st = alloc_orbitals(c, b))) return st;
    PARO_CU(c, cudaMemcpyAsync(dmap, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PARO_CU(c, cudaMemsetAsync(b.d_psi, 0, (size_t)c->nb * b.npw * sizeof(double2), c->stream));
    k_prolong<<<dim3((old_npw[ik] + 255) / 256, c->nb), 256, 0, c->stream>>>(old_npw[ik], b.npw, dmap, old_psi[ik],
                                                                           b.d_psi);
    PARO_LAUNCH(c, "k_prolong");
    PARO_CU(c, cudaStreamSynchronize(c->stream));
    cudaFree(old_psi[ik]);
    old_psi[ik] = nullptr;
    b.eps = old_eps[ik];
    if (c->have_veff && (st = adopt_orbitals(c, ik))) return st;
  }
  return PARO_OK;
}

// ================================================================================================
// C ABI
// ================================================================================================
#define CTX_CHECK(ctx)                                       \
  if (!(ctx)) return PARO_ERR_ARG;                           \
  Ctx* c = &(ctx)->c;                                        \
  c->err.clear();

extern "C" {

int paro_create(paro_ctx** out, const double lattice[9], int n_atoms, const double* pos, double ecut_ha, int n_k,
                const double* k_frac, const double* k_w, int n_bands, int n_occ, int precision, void* stream) {
  g_create_err.clear();
  if (!out || !lattice || n_atoms < 0 || (n_atoms > 0 && !pos) || !(ecut_ha > 0) || n_k < 1 ||
      (n_k > 1 && !k_frac) || n_bands < 1 || n_occ < 0 || n_occ > n_bands ||
      (precision != PARO_FP64 && precision != PARO_MIXED)) {
    g_create_err = "paro_create: invalid argument";
    return PARO_ERR_ARG;
  }
  *out = nullptr;
  paro_ctx* ctx = new paro_ctx;
  Ctx* c = &ctx->c;
  auto bail = [&](int code) {
    g_create_err = c->err.empty() ? "paro_create failed" : c->err;
    paro_destroy(ctx);
    return code;
  };
  for (int i = 0; i < 9; ++i) c->lat[i] = lattice[i];
  const double* L = c->lat;
  const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                     L[2] * (L[3] * L[7] - L[4] * L[6]);
  if (!(std::fabs(det) > 1e-12)) {
    c->err = "paro_create: singular lattice";
    return bail(PARO_ERR_ARG);
  }
  c->omega = std::fabs(det);
  // b_i = 2 pi (a_j x a_k) / det
  for (int i = 0; i < 3; ++i) {
    const double* u = L + 3 * ((i + 1) % 3);
    const double* v = L + 3 * ((i + 2) % 3);
    c->bmat[3 * i + 0] = 2 * kPi * (u[1] * v[2] - u[2] * v[1]) / det;
    c->bmat[3 * i + 1] = 2 * kPi * (u[2] * v[0] - u[0] * v[2]) / det;
    c->bmat[3 * i + 2] = 2 * kPi * (u[0] * v[1] - u[1] * v[0]) / det;
  }
  c->nat = n_atoms;
  c->pos.assign(pos, pos + 3 * n_atoms);
  c->ecut = ecut_ha;
  c->nk = n_k;
  c->nb = n_bands;
  c->nocc = n_occ;
  c->prec = precision;
  c->kw.resize(n_k);
  double wsum = 0;
  for (int i = 0; i < n_k; ++i) wsum += (c->kw[i] = k_w ? k_w[i] : 1.0 / n_k);
  if (!(std::fabs(wsum - 1.0) < 1e-8)) {
    c->err = "paro_create: k-point weights must sum to 1";
    return bail(PARO_ERR_ARG);
  }
  c->stream = static_cast<cudaStream_t>(stream);  // NULL: the default stream
  c->own_stream = false;
  // bases and the FFT grid of the cutoff
  c->bases.resize(n_k);
  for (int ik = 0; ik < n_k; ++ik) {
    Basis& b = c->bases[ik];
    for (int i = 0; i < 3; ++i) b.kfrac[i] = k_frac ? k_frac[3 * ik + i] : 0.0;
    for (int x = 0; x < 3; ++x)
      b.kcart[x] = b.kfrac[0] * c->bmat[x] + b.kfrac[1] * c->bmat[3 + x] + b.kfrac[2] * c->bmat[6 + x];
  }
  if (int st = setup_bases(c)) {
    c->err = "paro_create: " + (c->err.empty() ? std::string("basis setup failed") : c->err);
    return bail(st);
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(PARO_ERR_CUDA);
  *out = ctx;
  return PARO_OK;
}

void paro_destroy(paro_ctx* ctx) {
  if (!ctx) return;
  Ctx* c = &ctx->c;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (Basis& b : c->bases) free_basis(b);
  void* ps[] = {c->d_tw64[0], c->d_tw64[1], c->d_tw64[2], c->d_tw32[0], c->d_tw32[1], c->d_tw32[2],
                c->d_vloc, c->d_dvec, c->d_dvec32, c->d_veff, c->d_vplane, c->d_vplane32,
                c->d_rho_in, c->d_pulay_rho, c->d_pulay_res, c->d_pulay_gram, c->d_tc_err, c->d_occ_sqrt};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (auto& kv : c->ws) cudaFree(kv.second.first);
  for (auto& e : c->prof_ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  for (auto& kv : c->pinned) {
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    if (kv.second.h) cudaFreeHost(kv.second.h);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete ctx;
}

const char* paro_last_error(const paro_ctx* ctx) { return ctx ? ctx->c.err.c_str() : g_create_err.c_str(); }

int paro_grid(const paro_ctx* ctx, int n[3]) {
  if (!ctx || !n) return PARO_ERR_ARG;
  for (int i = 0; i < 3; ++i) n[i] = ctx->c.N[i];
  return PARO_OK;
}

int paro_npw(const paro_ctx* ctx, int ik, int* npw) {
  if (!ctx || !npw || ik < 0 || ik >= ctx->c.nk) return PARO_ERR_ARG;
  *npw = ctx->c.bases[ik].npw;
  return PARO_OK;
}

int paro_miller(const paro_ctx* ctx, int ik, int* hkl) {
  if (!ctx || !hkl || ik < 0 || ik >= ctx->c.nk) return PARO_ERR_ARG;
  const Basis& b = ctx->c.bases[ik];
  std::memcpy(hkl, b.miller.data(), b.miller.size() * sizeof(int));
  return PARO_OK;
}

int paro_sigma(const paro_ctx* ctx, double* sigma) {
  if (!ctx || !sigma) return PARO_ERR_ARG;
  if (!ctx->c.have_veff) return PARO_ERR_STATE;
  Ctx* c = const_cast<Ctx*>(&ctx->c);  // completes the pending read-back of the potential's minimum
  int st = veff_stats(c);
  if (st) return st;
  *sigma = c->sigma_k[0];
  return PARO_OK;
}

int paro_set_local_pp(paro_ctx* ctx, double Z, double rc, double A, double a) {
  CTX_CHECK(ctx);
  if (!(rc > 0) || !(a > 0)) return fail(c, PARO_ERR_ARG, "rc and a must be positive");
  c->Z = Z; c->rc = rc; c->A = A; c->a = a;
  int st = build_vloc(c);
  if (st) return st;
  c->have_pp = true;
  c->e_ewald = ewald(c);
  if ((st = set_veff_device(c, c->d_vloc))) return st;
  return PARO_OK;
}

int paro_set_kb(paro_ctx* ctx, double rc, const double* D) {
  CTX_CHECK(ctx);
  if (!(rc > 0) || !D) return fail(c, PARO_ERR_ARG, "bad KB arguments");
  c->kb_rc = rc;
  c->D.assign(D, D + 2 * c->nat);
  int st = build_beta(c);
  if (st) return st;
  std::vector<double> dv(c->nproj);
  for (int I = 0; I < c->nat; ++I) {
    dv[4 * I] = D[2 * I];
    dv[4 * I + 1] = dv[4 * I + 2] = dv[4 * I + 3] = D[2 * I + 1];
  }
  if (!c->d_dvec) PARO_CU(c, cudaMalloc(&c->d_dvec, std::max(c->nproj, 1) * sizeof(double)));
  PARO_CU(c, cudaMemcpy(c->d_dvec, dv.data(), c->nproj * sizeof(double), cudaMemcpyHostToDevice));
  c->have_kb = c->nproj > 0;
  return PARO_OK;
}

int paro_set_positions(paro_ctx* ctx, const double* pos) {
  CTX_CHECK(ctx);
  if (c->nat > 0 && !pos) return fail(c, PARO_ERR_ARG, "paro_set_positions: null positions");
  int st;
  double* v = nullptr;
  if (c->have_veff) {  // keep V_eff - V_loc
    v = static_cast<double*>(ws_get(c, "grid_r1", (size_t)c->ngrid * sizeof(double)));
    if (!v) return PARO_ERR_CUDA;
    PARO_CU(c, cudaMemcpyAsync(v, c->d_veff, (size_t)c->ngrid * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
    if (c->have_pp) {
      k_axpy_grid<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, -1.0, c->d_vloc, v);
      PARO_LAUNCH(c, "k_axpy_grid");
    }
  }
  c->pos.assign(pos, pos + 3 * c->nat);
  if (c->have_pp) {
    if ((st = build_vloc(c))) return st;
    c->e_ewald = ewald(c);
  }
  if (c->have_kb && (st = build_beta(c))) return st;
  if (v) {
    if (c->have_pp) {
      k_axpy_grid<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, 1.0, c->d_vloc, v);
      PARO_LAUNCH(c, "k_axpy_grid");
    }
    if ((st = set_veff_device(c, v))) return st;
  }
  for (int ik = 0; ik < c->nk; ++ik)
    if (c->bases[ik].have_psi && (st = reproject(c, ik))) return st;
  return PARO_OK;
}

int paro_set_veff(paro_ctx* ctx, const double* v_r, int on_device) {
  CTX_CHECK(ctx);
  if (!v_r) return fail(c, PARO_ERR_ARG, "null potential");
  double* tmp = static_cast<double*>(ws_get(c, "grid_r1", (size_t)c->ngrid * sizeof(double)));
  if (!tmp) return PARO_ERR_CUDA;
  PARO_CU(c, cudaMemcpyAsync(tmp, v_r, (size_t)c->ngrid * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  int st = set_veff_device(c, tmp);
  if (st) return st;
  return PARO_OK;
}

int paro_set_veff_rest(paro_ctx* ctx, const double* v_rest, int on_device) {
  CTX_CHECK(ctx);
  if (!v_rest) return fail(c, PARO_ERR_ARG, "null potential");
  if (!c->have_pp) return fail(c, PARO_ERR_STATE, "paro_set_veff_rest: no local pseudopotential");
  double* tmp = static_cast<double*>(ws_get(c, "grid_r1", (size_t)c->ngrid * sizeof(double)));
  if (!tmp) return PARO_ERR_CUDA;
  PARO_CU(c, cudaMemcpyAsync(tmp, v_rest, (size_t)c->ngrid * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  k_axpy_grid<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, 1.0, c->d_vloc, tmp);
  PARO_LAUNCH(c, "k_axpy_grid");
  int st = set_veff_device(c, tmp);
  if (st) return st;
  return PARO_OK;
}

int paro_get_veff(paro_ctx* ctx, double* v_r) {
  CTX_CHECK(ctx);
  if (!v_r) return PARO_ERR_ARG;
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no potential");
  PARO_CU(c, cudaMemcpyAsync(v_r, c->d_veff, (size_t)c->ngrid * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  return PARO_OK;
}

int paro_get_vloc(paro_ctx* ctx, double* v_r) {
  CTX_CHECK(ctx);
  if (!v_r) return PARO_ERR_ARG;
  if (!c->have_pp) return fail(c, PARO_ERR_STATE, "no local pseudopotential");
  PARO_CU(c, cudaMemcpyAsync(v_r, c->d_vloc, (size_t)c->ngrid * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  return PARO_OK;
}

int paro_set_density(paro_ctx* ctx, const double* rho, int on_device) {
  CTX_CHECK(ctx);
  if (!rho) return PARO_ERR_ARG;
  if (!c->d_rho_in) PARO_CU(c, cudaMalloc(&c->d_rho_in, (size_t)c->ngrid * sizeof(double)));
  PARO_CU(c, cudaMemcpyAsync(c->d_rho_in, rho, (size_t)c->ngrid * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  int st = veff_from_density(c, c->d_rho_in, nullptr, nullptr);
  if (st) return st;
  c->have_rho = true;
  return PARO_OK;
}

int paro_set_ecut(paro_ctx* ctx, double ecut_ha) {
  CTX_CHECK(ctx);
  if (!std::isfinite(ecut_ha) || ecut_ha < c->ecut)
    return fail(c, PARO_ERR_ARG, "paro_set_ecut: the cutoff ladder only raises E_cut");
  if (ecut_ha == c->ecut) return PARO_OK;
  const double old = c->ecut;
  int st = set_ecut(c, ecut_ha);
  if (st && c->ecut != old && c->err.empty()) c->err = "paro_set_ecut failed";
  return st;
}

int paro_set_gamma_real(paro_ctx* ctx, int enable) {
  CTX_CHECK(ctx);
  if (!enable) {
    c->gamma_real = false;
    return PARO_OK;
  }
  const Basis& b0 = c->bases[0];
  if (c->nk != 1 || b0.kfrac[0] != 0 || b0.kfrac[1] != 0 || b0.kfrac[2] != 0)
    return fail(c, PARO_ERR_ARG, "paro_set_gamma_real: the real-wavefunction mode needs the Gamma point only");
  int st = gamma_build_table(c, 0);
  if (st) return st;
  c->gamma_real = true;
  if (c->bases[0].have_psi) {  // the current orbitals become real and take their Ritz pairs again
    if ((st = fp64_current(c, c->bases[0]))) return st;
    if ((st = gamma_real_rows<double>(c, 0, c->nb, c->bases[0].d_psi))) return st;
    if ((st = reproject(c, 0))) return st;
  }
  return PARO_OK;
}

int paro_set_smearing(paro_ctx* ctx, double kT) {
  CTX_CHECK(ctx);
  if (!(kT >= 0) || !std::isfinite(kT)) return fail(c, PARO_ERR_ARG, "paro_set_smearing: kT must be >= 0");
  c->kT = kT;
  return PARO_OK;
}

int paro_get_occupations(paro_ctx* ctx, double* f, double* mu, double* minus_ts) {
  CTX_CHECK(ctx);
  for (int ik = 0; ik < c->nk; ++ik)
    if (!c->bases[ik].have_psi) return fail(c, PARO_ERR_STATE, "no orbitals");
  int st = update_occupations(c);
  if (st) return st;
  if (f) std::copy(c->occ.begin(), c->occ.end(), f);
  if (mu) *mu = c->mu;
  if (minus_ts) *minus_ts = c->mts;
  return PARO_OK;
}

int paro_apply_h(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, void* hpsi) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || nb < 1 || !psi || !hpsi || psi == hpsi ||
      (dtype != PARO_C64 && dtype != PARO_C32))
    return fail(c, PARO_ERR_ARG, "paro_apply_h: bad argument");
  if (dtype == PARO_C64 && check_fft_support(c, 16)) return PARO_ERR_ARG;
  GammaPackOff general(c);  // the caller's vectors are general complex rows
  return dtype == PARO_C64
             ? apply_h<double>(c, ik, nb, static_cast<const double2*>(psi), static_cast<double2*>(hpsi), 0.0, nullptr)
             : apply_h<float>(c, ik, nb, static_cast<const float2*>(psi), static_cast<float2*>(hpsi), 0.0, nullptr);
}

int paro_apply_vnl(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, void* out, int form) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || nb < 1 || !psi || !out || psi == out || (dtype != PARO_C64 && dtype != PARO_C32) ||
      (form != PARO_VNL_ACCURATE && form != PARO_VNL_TENSOR) || (form == PARO_VNL_TENSOR && dtype != PARO_C32))
    return fail(c, PARO_ERR_ARG, "paro_apply_vnl: bad argument");
  if (!c->have_kb) return fail(c, PARO_ERR_STATE, "paro_apply_vnl: no Kleinman-Bylander projectors set");
  const size_t eb = dtype == PARO_C64 ? sizeof(double2) : sizeof(float2);
  PARO_CU(c, cudaMemsetAsync(out, 0, (size_t)nb * c->bases[ik].npw * eb, c->stream));
  int st;
  if (dtype == PARO_C64) {
    st = kb_apply<double>(c, ik, nb, static_cast<const double2*>(psi), static_cast<double2*>(out));
  } else if (form == PARO_VNL_TENSOR) {
    TcScope tcs(c);
    st = kb_apply<float>(c, ik, nb, static_cast<const float2*>(psi), static_cast<float2*>(out));
  } else {
    st = kb_apply<float>(c, ik, nb, static_cast<const float2*>(psi), static_cast<float2*>(out));
  }
  if (st) return st;
  const int* htc = nullptr;
  if ((st = tc_flag_readback(c, &htc))) return st;
  if (htc) {
    if ((st = pinned_wait(c, "tc_err"))) return st;
    if (*htc) return fail(c, PARO_ERR_TIMEOUT, "tensor-core product: mbarrier wait gave up");
  }
  return PARO_OK;
}

int paro_apply_h_adjoint(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, const void* w, void* g_psi,
                         double* g_v, double* g_pos) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || nb < 1 || !psi || !w || (dtype != PARO_C64 && dtype != PARO_C32) ||
      g_psi == psi || g_psi == w)
    return fail(c, PARO_ERR_ARG, "paro_apply_h_adjoint: bad argument");
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no effective potential set");
  if (dtype == PARO_C64 && check_fft_support(c, 16)) return PARO_ERR_ARG;
  GammaPackOff general(c);
  return apply_h_adjoint(c, ik, nb, dtype, psi, w, g_psi, g_v, g_pos);
}

int paro_orthonormalize(paro_ctx* ctx, int ik, int n, int dtype, const void* x, void* y) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || n < 1 || !x || !y || (dtype != PARO_C64 && dtype != PARO_C32))
    return fail(c, PARO_ERR_ARG, "paro_orthonormalize: bad argument");
  const int npw = c->bases[ik].npw;
  if (n > npw) return fail(c, PARO_ERR_ARG, "paro_orthonormalize: more rows than plane waves");
  const size_t bytes = (size_t)n * npw * (dtype == PARO_C64 ? sizeof(double2) : sizeof(float2));
  const char *xb = static_cast<const char*>(x), *yb = static_cast<const char*>(y);
  if (x != y && xb < yb + bytes && yb < xb + bytes) return fail(c, PARO_ERR_ARG, "paro_orthonormalize: x and y overlap");
  if (x != y) PARO_CU(c, cudaMemcpyAsync(y, x, bytes, cudaMemcpyDeviceToDevice, c->stream));
  GammaPackOff general(c);
  return dtype == PARO_C64 ? orthonormalize<double>(c, ik, static_cast<double2*>(y), n)
                           : orthonormalize<float>(c, ik, static_cast<float2*>(y), n);
}

int paro_solve_source(paro_ctx* ctx, int ik, int nb, int dtype, const double* eps, const void* psi, void* x,
                      double rel_tol, int max_it, int* iters_out) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || nb < 1 || !eps || !psi || !x || psi == x || max_it < 0 ||
      (dtype != PARO_C64 && dtype != PARO_C32))
    return fail(c, PARO_ERR_ARG, "paro_solve_source: bad argument");
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no effective potential set");
  GammaPackOff general(c);
  const int npw = c->bases[ik].npw;
  double* f = static_cast<double*>(ws_get(c, "ss_f", (size_t)nb * sizeof(double)));
  if (!f) return PARO_ERR_CUDA;
  int st0 = veff_stats(c);
  if (st0) return st0;
  std::vector<double> hf(nb);
  for (int i = 0; i < nb; ++i) hf[i] = eps[i] - c->sigma_k[ik];
  if ((st0 = h2d_async(c, "ss_f", f, hf.data(), nb * sizeof(double)))) return st0;
  if (dtype == PARO_C64) {
    double2* rhs = static_cast<double2*>(ws_get(c, "src_rhs64", (size_t)nb * npw * sizeof(double2)));
    if (!rhs) return PARO_ERR_CUDA;
    int st = scale_rows<double>(c, nb, npw, static_cast<const double2*>(psi), f, rhs);
    if (st) return st;
    PARO_CU(c, cudaMemcpyAsync(x, psi, (size_t)nb * npw * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    return pcg_run<double>(c, ik, nb, rhs, static_cast<double2*>(x), false, rel_tol, max_it, iters_out);
  }
  float2* rhs = static_cast<float2*>(ws_get(c, "src_rhs32", (size_t)nb * npw * sizeof(float2)));
  if (!rhs) return PARO_ERR_CUDA;
  int st = scale_rows<float>(c, nb, npw, static_cast<const float2*>(psi), f, rhs);
  if (st) return st;
  PARO_CU(c, cudaMemcpyAsync(x, psi, (size_t)nb * npw * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
  return pcg_run<float>(c, ik, nb, rhs, static_cast<float2*>(x), false, rel_tol, max_it, iters_out);
}

int paro_set_orbitals(paro_ctx* ctx, int ik, const void* psi, int on_device) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || !psi) return fail(c, PARO_ERR_ARG, "paro_set_orbitals: bad argument");
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no effective potential set");
  Basis& b = c->bases[ik];
  int st = alloc_orbitals(c, b);
  if (st) return st;
  PARO_CU(c, cudaMemcpyAsync(b.d_psi, psi, (size_t)c->nb * b.npw * sizeof(double2),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  if (c->gamma_real && (st = gamma_real_rows<double>(c, ik, c->nb, b.d_psi))) return st;
  return reproject(c, ik);
}

int paro_get_orbitals(paro_ctx* ctx, int ik, void* psi, int on_device) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || !psi) return PARO_ERR_ARG;
  Basis& b = c->bases[ik];
  if (!b.have_psi) return fail(c, PARO_ERR_STATE, "no orbitals");
  if (int st = fp64_current(c, b)) return st;
  PARO_CU(c, cudaMemcpyAsync(psi, b.d_psi, (size_t)c->nb * b.npw * sizeof(double2),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  return PARO_OK;
}

int paro_get_eigenvalues(paro_ctx* ctx, double* eps) {
  CTX_CHECK(ctx);
  if (!eps) return PARO_ERR_ARG;
  for (int ik = 0; ik < c->nk; ++ik) {
    if (!c->bases[ik].have_psi) return fail(c, PARO_ERR_STATE, "no orbitals");
    std::copy(c->bases[ik].eps.begin(), c->bases[ik].eps.end(), eps + (size_t)ik * c->nb);
  }
  return PARO_OK;
}

int paro_get_residuals(paro_ctx* ctx, double* res) {
  CTX_CHECK(ctx);
  if (!res) return PARO_ERR_ARG;
  for (int ik = 0; ik < c->nk; ++ik) {
    if (!c->bases[ik].have_psi) return fail(c, PARO_ERR_STATE, "no orbitals");
    if (int st = project_readback(c, ik)) return st;
    std::copy(c->bases[ik].res.begin(), c->bases[ik].res.end(), res + (size_t)ik * c->nb);
  }
  return PARO_OK;
}

int paro_step(paro_ctx* ctx, int alg, double rel_tol, int max_it, double* max_resid_out) {
  CTX_CHECK(ctx);
  if ((alg != PARO_ALG1 && alg != PARO_ALG2 && alg != PARO_ALG3) || max_it < 0)
    return fail(c, PARO_ERR_ARG, "paro_step: bad argument");
  for (int ik = 0; ik < c->nk; ++ik) {
    if (!c->bases[ik].have_psi) return fail(c, PARO_ERR_STATE, "paro_step: orbitals not set");
    int st = c->prec == PARO_MIXED ? paro_step_k<float>(c, ik, alg, rel_tol, max_it)
                                   : paro_step_k<double>(c, ik, alg, rel_tol, max_it);
    if (st) return st;
  }
  if (max_resid_out) *max_resid_out = max_occ_resid(c);
  return PARO_OK;
}

int paro_eigh(paro_ctx* ctx, int n, const void* a, double* w, void* v) {
  CTX_CHECK(ctx);
  if (n < 1 || !a || !w || !v) return fail(c, PARO_ERR_ARG, "paro_eigh: bad argument");
  return c->prec == PARO_MIXED ? eigh_mixed(c, n, static_cast<const double2*>(a), w, static_cast<double2*>(v), 2)
                               : eigh(c, n, static_cast<const double2*>(a), w, static_cast<double2*>(v));
}

int paro_density(paro_ctx* ctx, double* rho_dev) {
  CTX_CHECK(ctx);
  if (!rho_dev) return PARO_ERR_ARG;
  for (int ik = 0; ik < c->nk; ++ik)
    if (!c->bases[ik].have_psi) return fail(c, PARO_ERR_STATE, "no orbitals");
  return current_density(c, rho_dev);
}

int paro_energy(paro_ctx* ctx, double terms[7]) {
  CTX_CHECK(ctx);
  if (!terms) return PARO_ERR_ARG;
  if (!c->have_pp) return fail(c, PARO_ERR_STATE, "no local pseudopotential");
  double* rho = static_cast<double*>(ws_get(c, "energy_rho", (size_t)c->ngrid * sizeof(double)));
  if (!rho) return PARO_ERR_CUDA;
  int st = paro_density(ctx, rho);
  if (st) return st;
  return energy_terms(c, rho, terms);
}

__global__ void k_fill(int n, double v, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

int paro_scf_step(paro_ctx* ctx, const paro_scf_opts* o, double energy[7], double* max_resid_out) {
  CTX_CHECK(ctx);
  if (!o || (o->alg != PARO_ALG1 && o->alg != PARO_ALG2 && o->alg != PARO_ALG3))
    return fail(c, PARO_ERR_ARG, "paro_scf_step: bad options");
  if (!c->have_pp) return fail(c, PARO_ERR_STATE, "no local pseudopotential");
  for (int ik = 0; ik < c->nk; ++ik)
    if (!c->bases[ik].have_psi) return fail(c, PARO_ERR_STATE, "orbitals not set");
  int st;
  if (!c->have_rho) {  // first iteration: uniform density, Ritz pairs of the start span under its potential
    if (!c->d_rho_in) PARO_CU(c, cudaMalloc(&c->d_rho_in, (size_t)c->ngrid * sizeof(double)));
    k_fill<<<(c->ngrid + 255) / 256, 256, 0, c->stream>>>(c->ngrid, 2.0 * c->nocc / c->omega, c->d_rho_in);
    PARO_LAUNCH(c, "k_fill");
    if ((st = veff_from_density(c, c->d_rho_in, nullptr, nullptr))) return st;
      for (int ik = 0; ik < c->nk; ++ik)
      if ((st = reproject(c, ik))) return st;
    c->have_rho = true;
    c->scf_iter = 0;
    c->scf_small = 0;
    c->pulay_n = 0;
    c->pulay_head = 0;
  }
  st = c->prec == PARO_MIXED ? scf_iteration<float>(c, o) : scf_iteration<double>(c, o);
  if (st) return st;
  double terms[7];
  {
    ProfTag t(c, "energy");
    if ((st = paro_energy(ctx, terms))) return st;
  }
  if (energy) std::copy(terms, terms + 7, energy);
  for (int ik = 0; ik < c->nk; ++ik)
    if ((st = project_readback(c, ik))) return st;
  if (max_resid_out) *max_resid_out = max_occ_resid(c);
  const double e = terms[PARO_E_TOTAL];
  if (c->scf_iter > 0 && std::fabs(e - c->e_prev) / std::max(c->nat, 1) < o->tol_per_atom)
    ++c->scf_small;
  else
    c->scf_small = 0;
  c->e_prev = e;
  ++c->scf_iter;
  return PARO_OK;
}

int paro_set_state(paro_ctx* ctx, int ik, const void* psi, const double* eps, int on_device) {
  CTX_CHECK(ctx);
  if (ik < 0 || ik >= c->nk || !psi || !eps) return fail(c, PARO_ERR_ARG, "paro_set_state: bad argument");
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no effective potential set");
  Basis& b = c->bases[ik];
  int st = alloc_orbitals(c, b);
  if (st) return st;
  const size_t bytes = (size_t)c->nb * b.npw * sizeof(double2);
  PARO_CU(c, cudaMemcpyAsync(b.d_psi, psi, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
  if (c->gamma_real && (st = gamma_real_rows<double>(c, ik, c->nb, b.d_psi))) return st;
  b.eps.assign(eps, eps + c->nb);
  return adopt_orbitals(c, ik);
}

int paro_profile(paro_ctx* ctx, int enable) {
  CTX_CHECK(ctx);
  cudaStreamSynchronize(c->stream);
  for (auto& e : c->prof_ev) {
    c->prof_pool.push_back(e.a);
    c->prof_pool.push_back(e.b);
  }
  c->prof_ev.clear();
  c->prof = enable != 0;
  while (c->prof && c->prof_pool.size() < 512) {  // created here, not inside the recorded region
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) break;
    c->prof_pool.push_back(e);
  }
  return PARO_OK;
}

int paro_profile_read(paro_ctx* ctx, const char* name, int* count, double* total_ms) {
  CTX_CHECK(ctx);
  if (!name || !count || !total_ms) return PARO_ERR_ARG;
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  int n = 0;
  double t = 0;
  for (auto& e : c->prof_ev) {
    if (e.name != name && std::strcmp(name, "*") != 0) continue;
    float ms = 0;
    PARO_CU(c, cudaEventElapsedTime(&ms, e.a, e.b));
    ++n;
    t += ms;
  }
  *count = n;
  *total_ms = t;
  return PARO_OK;
}

int paro_profile_names(paro_ctx* ctx, char* buf, int len) {
  CTX_CHECK(ctx);
  if (!buf || len < 1) return PARO_ERR_ARG;
  std::vector<std::string> names;
  for (auto& e : c->prof_ev)
    if (std::find(names.begin(), names.end(), e.name) == names.end()) names.push_back(e.name);
  std::string s;
  for (auto& n : names) s += (s.empty() ? "" : ",") + n;
  std::strncpy(buf, s.c_str(), len - 1);
  buf[len - 1] = 0;
  return PARO_OK;
}

int paro_launch_count(const paro_ctx* ctx, long long* n) {
  if (!ctx || !n) return PARO_ERR_ARG;
  *n = ctx->c.launches;
  return PARO_OK;
}

int paro_scf(paro_ctx* ctx, const paro_scf_opts* o, paro_scf_result* r) {
  CTX_CHECK(ctx);
  if (!o || !r || o->max_iter < 1) return fail(c, PARO_ERR_ARG, "paro_scf: bad argument");
  std::memset(r, 0, sizeof(*r));
  for (int it = 0; it < o->max_iter; ++it) {
    int st = paro_scf_step(ctx, o, r->energy, &r->max_resid);
    if (st) return st;
    r->n_iter = it + 1;
    if (c->scf_small >= 2) {
      r->converged = 1;
      return PARO_OK;
    }
  }
  return fail(c, PARO_ERR_NOT_CONVERGED, "SCF did not converge within max_iter");
}

}  // extern "C"
