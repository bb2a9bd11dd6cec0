// H psi for a batch of orbitals (Eq. e5 applied through the FFT), three passes over the FFT grid:
//
//   pass 1  scatter each z-column ("stick") of the cutoff sphere into a line of N3 points and
//           inverse-FFT it along z; sticks of one band are written plane-major S[b][z][stick];
//   pass 2  per (band, z-plane): place the plane's sticks on the N1 x N2 plane, inverse-FFT along y
//           (only the rows that hold sticks) and along x, multiply by V_eff(r)/N_grid, forward-FFT
//           along x and along y (rows with sticks only), and keep the stick positions;
//   pass 3  forward-FFT each stick along z and gather the sphere coefficients, adding the kinetic
//           term |k+G|^2/2 c_G (and an optional shift -sigma c_G for the PCG operator H - sigma).
//
// The nonlocal Kleinman-Bylander part (Section 2.2, V_nl) is added afterwards by two GEMMs:
// P = beta^H psi (nproj x nb), then H psi += beta (D o P).
#include <mutex>

#include "fft_reg.cuh"
#include "paro_ctx.h"

namespace paro {

// ------------------------------------------------------------------------------------------------
// pass 1
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, 2) k_zpass_inv(const cplx<T>* __restrict__ psi, int ldpsi,
                                                   cplx<T>* __restrict__ S, const int* __restrict__ col_off,
                                                   const int* __restrict__ g_col, const int* __restrict__ g_z,
                                                   int ncol, FftPlan pz, const cplx<T>* __restrict__ twz,
                                                   const int* __restrict__ active, int CB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  const int N3 = pz.n, ls = N3 + 1;
  cplx<T>* line = tw + N3;
  const int b = blockIdx.y;
  if (active != nullptr && active[b] == 0) return;
  const int c0 = blockIdx.x * CB;
  const int ncb = min(CB, ncol - c0);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) tw[i] = twz[i];
  for (int i = threadIdx.x; i < ncb * ls; i += blockDim.x) line[i] = mk<T>(0, 0);
  __syncthreads();
  const int g0 = col_off[c0], g1 = col_off[c0 + ncb];
  const cplx<T>* p = psi + (size_t)b * ldpsi;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) line[(g_col[g] - c0) * ls + g_z[g]] = p[g];
  __syncthreads();
  fft_lines<T, true, false>(line, pz, ncb, 1, LinesDirect{ls}, tw);
  cplx<T>* Sb = S + (size_t)b * N3 * ncol;
  for (int i = threadIdx.x; i < N3 * ncb; i += blockDim.x) {
    const int z = i / ncb, cc = i - z * ncb;
    Sb[(size_t)z * ncol + c0 + cc] = line[cc * ls + z];
  }
}

// ------------------------------------------------------------------------------------------------
// pass 2
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512, 1) k_plane(cplx<T>* __restrict__ S, int ncol, const int* __restrict__ col_x,
                        const int* __restrict__ col_y, const int* __restrict__ xrows, int nxr, FftPlan px,
                        FftPlan py, const cplx<T>* __restrict__ twx, const cplx<T>* __restrict__ twy,
                        const T* __restrict__ vplane, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N1 = px.n, N2 = py.n;
  cplx<T>* tx = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* ty = tx + N1;
  cplx<T>* P = ty + N2;
  const int z = blockIdx.x, b = blockIdx.y, N3 = gridDim.x;
  if (active != nullptr && active[b] == 0) return;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) P[i] = mk<T>(0, 0);
  __syncthreads();
  cplx<T>* Sz = S + ((size_t)b * N3 + z) * ncol;
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) P[col_x[c] * N2 + col_y[c]] = Sz[c];
  __syncthreads();
  fft_lines<T, true, false>(P, py, nxr, 1, LinesMapped{xrows, N2}, ty);
  fft_lines<T, true, true>(P, px, N2, N2, LinesDirect{1}, tx);
  const T* V = vplane + (size_t)z * N1 * N2;
  for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) P[i] = cscale(P[i], V[i]);
  __syncthreads();
  fft_lines<T, false, true>(P, px, N2, N2, LinesDirect{1}, tx);
  fft_lines<T, false, false>(P, py, nxr, 1, LinesMapped{xrows, N2}, ty);
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) Sz[c] = P[col_x[c] * N2 + col_y[c]];
}

// ------------------------------------------------------------------------------------------------
// pass 3
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, 2) k_zpass_fwd(const cplx<T>* __restrict__ S, const cplx<T>* __restrict__ psi,
                                                   int ldpsi, cplx<T>* __restrict__ hpsi, int ldh,
                                                   const T* __restrict__ kin, T shift,
                                                   const int* __restrict__ col_off, const int* __restrict__ g_col,
                                                   const int* __restrict__ g_z, int ncol, FftPlan pz,
                                                   const cplx<T>* __restrict__ twz,
                                                   const int* __restrict__ active, int CB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  const int N3 = pz.n, ls = N3 + 1;
  cplx<T>* line = tw + N3;
  const int b = blockIdx.y;
  if (active != nullptr && active[b] == 0) return;
  const int c0 = blockIdx.x * CB;
  const int ncb = min(CB, ncol - c0);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) tw[i] = twz[i];
  const cplx<T>* Sb = S + (size_t)b * N3 * ncol;
  for (int i = threadIdx.x; i < N3 * ncb; i += blockDim.x) {
    const int z = i / ncb, cc = i - z * ncb;
    line[cc * ls + z] = Sb[(size_t)z * ncol + c0 + cc];
  }
  __syncthreads();
  fft_lines<T, false, false>(line, pz, ncb, 1, LinesDirect{ls}, tw);
  const int g0 = col_off[c0], g1 = col_off[c0 + ncb];
  const cplx<T>* p = psi + (size_t)b * ldpsi;
  cplx<T>* h = hpsi + (size_t)b * ldh;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const cplx<T> v = line[(g_col[g] - c0) * ls + g_z[g]];
    const cplx<T> c = p[g];
    const T t = kin[g] - shift;
    h[g] = mk<T>(v.x + t * c.x, v.y + t * c.y);
  }
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
static const int kStickBatch = 32;
static const int kZThreads = 256;

static int plane_threads(const Ctx*) { return 512; }

// every stage must hold at least one whole line (lines are processed in groups)
static bool stages_fit(const FftPlan& p, int threads) {
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.rad[s];
    const int mu = R == 2 ? 4 : (R == 8 ? 1 : 2);
    if (p.n / R > mu * threads) return false;
  }
  return true;
}

static size_t zpass_smem(const Ctx* c, int eb) { return (size_t)eb * (c->N[2] + kStickBatch * (c->N[2] + 1)); }
static size_t plane_smem(const Ctx* c, int eb) { return (size_t)eb * (c->N[0] + c->N[1] + c->N[0] * c->N[1]); }

int check_fft_support(Ctx* c, int eb) {
  const int pt = plane_threads(c);
  if (!stages_fit(c->plan[2], kZThreads) || !stages_fit(c->plan[1], pt) || !stages_fit(c->plan[0], pt))
    return fail(c, PARO_ERR_ARG, "FFT grid too large for the register budget of the shared-memory FFT");
  if (plane_smem(c, eb) > 227 * 1024 || zpass_smem(c, eb) > 227 * 1024)
    return fail(c, PARO_ERR_ARG, "FFT plane does not fit in shared memory for this precision");
  return PARO_OK;
}

template <typename T>
static int configure(Ctx* c) {
  const int eb = (int)sizeof(cplx<T>);
  bool& d = c->fft_configured[sizeof(T) == 8];
  if (!d) {
    PARO_CU(c, cudaFuncSetAttribute(k_zpass_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    PARO_CU(c, cudaFuncSetAttribute(k_zpass_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    PARO_CU(c, cudaFuncSetAttribute(k_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    d = true;
  }
  return check_fft_support(c, eb);
}

template <typename T> static const cplx<T>* tw_of(const Ctx* c, int ax);
template <> const double2* tw_of<double>(const Ctx* c, int ax) { return c->d_tw64[ax]; }
template <> const float2* tw_of<float>(const Ctx* c, int ax) { return c->d_tw32[ax]; }
template <typename T> static const T* vplane_of(const Ctx* c);
template <> const double* vplane_of<double>(const Ctx* c) { return c->d_vplane; }
template <> const float* vplane_of<float>(const Ctx* c) { return c->d_vplane32; }
template <typename T> static const T* kin_of(const Basis& b);
template <> const double* kin_of<double>(const Basis& b) { return b.d_kin; }
template <> const float* kin_of<float>(const Basis& b) { return b.d_kin32; }

#include "hpsi_passes_reg.cuh"

template <typename T>
int apply_h(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi, double shift, const int* active) {
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no effective potential set");
  if (gamma_on(c)) return gamma_apply<T>(c, ik, nb, psi, hpsi, shift, active, nullptr, nullptr);
  int st = configure<T>(c);
  if (st) return st;
  const Basis& B = c->bases[ik];
  const int eb = (int)sizeof(cplx<T>);
  const size_t sbytes = (size_t)nb * c->N[2] * B.ncol * eb;
  cplx<T>* S = static_cast<cplx<T>*>(ws_get(c, sizeof(T) == 8 ? "sticks64" : "sticks32", sbytes));
  if (!S) return PARO_ERR_CUDA;
  bool used = false;
  if ((st = passes_reg_dispatch<T>(c, B, nb, psi, S, hpsi, shift, active, &used))) return st;
  if (used) {
    if (!c->have_kb) return PARO_OK;
    cudaEvent_t ev = prof_begin(c);
    st = kb_apply<T>(c, ik, nb, psi, hpsi);
    prof_end(c, sizeof(T) == 8 ? "kb_apply<f64>" : "kb_apply<f32>", ev);
    return st;
  }
  // shared-memory Stockham passes for the other grids
  const dim3 gz((B.ncol + kStickBatch - 1) / kStickBatch, nb);
  const bool f64 = sizeof(T) == 8;
  cudaEvent_t ev = prof_begin(c);
  k_zpass_inv<T><<<gz, kZThreads, zpass_smem(c, eb), c->stream>>>(psi, B.npw, S, B.d_col_off, B.d_g_col, B.d_g_z,
                                                                  B.ncol, c->plan[2], tw_of<T>(c, 2), active,
                                                                  kStickBatch);
  PARO_LAUNCH(c, "k_zpass_inv");
  prof_end(c, f64 ? "k_zpass_inv<f64>" : "k_zpass_inv<f32>", ev);
  ev = prof_begin(c);
  k_plane<T><<<dim3(c->N[2], nb), plane_threads(c), plane_smem(c, eb), c->stream>>>(
      S, B.ncol, B.d_col_x, B.d_col_y, B.d_xrows, B.nxr, c->plan[0], c->plan[1], tw_of<T>(c, 0), tw_of<T>(c, 1),
      vplane_of<T>(c), active);
  PARO_LAUNCH(c, "k_plane");
  prof_end(c, f64 ? "k_plane<f64>" : "k_plane<f32>", ev);
  ev = prof_begin(c);
  k_zpass_fwd<T><<<gz, kZThreads, zpass_smem(c, eb), c->stream>>>(S, psi, B.npw, hpsi, B.npw, kin_of<T>(B),
                                                                  (T)shift, B.d_col_off, B.d_g_col, B.d_g_z,
                                                                  B.ncol, c->plan[2], tw_of<T>(c, 2), active,
                                                                  kStickBatch);
  PARO_LAUNCH(c, "k_zpass_fwd");
  prof_end(c, f64 ? "k_zpass_fwd<f64>" : "k_zpass_fwd<f32>", ev);
  if (c->have_kb) {
    ev = prof_begin(c);
    int st2 = kb_apply<T>(c, ik, nb, psi, hpsi);
    prof_end(c, f64 ? "kb_apply<f64>" : "kb_apply<f32>", ev);
    return st2;
  }
  return PARO_OK;
}

// hpsi += dV psi for a change dV of the local potential (plane layout and scale of the context's V
// planes: dV / N_grid, [z][x][y]): the three FFT passes with dV in place of V, no kinetic or projector
// term. Register-FFT grids only; *used = false elsewhere (the caller applies H instead).
template <typename T>
int apply_dv(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi, const T* dvplane, bool* used) {
  *used = false;
  if (gamma_on(c)) return gamma_apply<T>(c, ik, nb, psi, hpsi, 0.0, nullptr, dvplane, used);
  int st = configure<T>(c);
  if (st) return st;
  const Basis& B = c->bases[ik];
  const size_t sbytes = (size_t)nb * c->N[2] * B.ncol * sizeof(cplx<T>);
  cplx<T>* S = static_cast<cplx<T>*>(ws_get(c, sizeof(T) == 8 ? "sticks64" : "sticks32", sbytes));
  if (!S) return PARO_ERR_CUDA;
  return passes_reg_dispatch<T>(c, B, nb, psi, S, hpsi, 0.0, nullptr, used, dvplane, true);
}
template int apply_dv<double>(Ctx*, int, int, const double2*, double2*, const double*, bool*);
template int apply_dv<float>(Ctx*, int, int, const float2*, float2*, const float*, bool*);

template <typename T>
int sticks_inverse(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* S) {
  int st = configure<T>(c);
  if (st) return st;
  bool used = false;
  if ((st = sticks_inverse_reg<T>(c, ik, nb, psi, S, &used)) || used) return st;
  const Basis& B = c->bases[ik];
  const dim3 gz((B.ncol + kStickBatch - 1) / kStickBatch, nb);
  k_zpass_inv<T><<<gz, kZThreads, zpass_smem(c, sizeof(cplx<T>)), c->stream>>>(
      psi, B.npw, S, B.d_col_off, B.d_g_col, B.d_g_z, B.ncol, c->plan[2], tw_of<T>(c, 2), nullptr, kStickBatch);
  PARO_LAUNCH(c, "k_zpass_inv");
  return PARO_OK;
}

template int sticks_inverse<double>(Ctx*, int, int, const double2*, double2*);
template int sticks_inverse<float>(Ctx*, int, int, const float2*, float2*);
template int density_planes_reg<double>(Ctx*, int, const double2*, int, int, int, double, const double*, double*,
                                         bool*, bool*);
template int density_planes_reg<float>(Ctx*, int, const float2*, int, int, int, double, const double*, double*,
                                        bool*, bool*);

template <typename T> static const cplx<T>* beta_of(const Basis& b);
template <> const double2* beta_of<double>(const Basis& b) { return b.d_beta; }
template <> const float2* beta_of<float>(const Basis& b) { return b.d_beta32; }

// H psi += beta (D o (beta^H psi))
template <typename T>
int kb_apply(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi) {
  const Basis& B = c->bases[ik];
  double2* P = static_cast<double2*>(ws_get(c, "kb_proj", (size_t)c->nproj * nb * sizeof(double2)));
  if (!P) return PARO_ERR_CUDA;
  // inside the inexact inner solves: the tensor-core products fed by the projectors' presplit images
  if constexpr (sizeof(T) == 4) {
    if (c->tc_scope && tc_enabled()) {
      int* err = tc_err_flag(c);
      if (!err) return PARO_ERR_CUDA;
      int st = beta_images(c, ik);
      if (st) return st;
      cudaEvent_t ev = prof_begin(c);
      if ((st = gemm_cn_tc_beta(c, ik, nb, reinterpret_cast<const float2*>(psi), P, err))) return st;
      prof_end(c, "k_gemm_cn_tcb", ev);
      ev = prof_begin(c);
      if ((st = gemm_wx_tc_beta(c, ik, nb, P, c->d_dvec, reinterpret_cast<float2*>(hpsi), err))) return st;
      prof_end(c, "k_gemm_wx_tcb", ev);
      return PARO_OK;
    }
  }
  // FP32 projections outside the inexact inner solves carry their sums in a two-sum pair: a long FP32
  // accumulation biases |<beta|psi>|^2 (and with it the Rayleigh-Ritz H and the energy) at the 1e-6 level
  const bool carry = sizeof(T) == 4 && !c->tc_scope;
  int st = gemm_cn<T, T, T>(c, c->nproj, nb, B.npw, beta_of<T>(B), B.npw, psi, B.npw, P, nb, false, carry);
  if (st) return st;
  // W(k = p, m = b) = D_p P[p][b]
  return gemm_wx<T, T>(c, nb, B.npw, c->nproj, P, nb, false, c->d_dvec, beta_of<T>(B), B.npw, hpsi, B.npw, 1.0);
}

template int apply_h<double>(Ctx*, int, int, const double2*, double2*, double, const int*);
template int apply_h<float>(Ctx*, int, int, const float2*, float2*, double, const int*);
template int kb_apply<double>(Ctx*, int, int, const double2*, double2*);
template int kb_apply<float>(Ctx*, int, int, const float2*, float2*);

// ------------------------------------------------------------------------------------------------
// Allocation-free H psi (paro_apply_h_noalloc). Some callers cannot let a library allocate device
// memory in the middle of their work: applications that hand all device memory to their own pool
// up front and run under a fixed budget, and callers that must not add the implicit device-wide
// synchronisation of cudaMalloc/cudaFree to a latency-critical loop. For them the stick buffer, the
// KB projections and the split-K partial sums of one H psi live in this file-scope device array,
// which every GPU that loads the library holds until the process exits.
// ------------------------------------------------------------------------------------------------
static const size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static const int kMaxDevices = 64;
static void* g_noalloc_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device. The symbol's name in host code is only
// a host-side stand-in, so the address is looked up once per device (with that device current) and
// cached; the first call on a device does this set-up.
static int noalloc_scratch(Ctx* c, unsigned char** out) {
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(c, PARO_ERR_ARG, "paro_apply_h_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return PARO_OK;
}

static size_t round256(size_t x) { return (x + 255) / 256 * 256; }

template <typename T>
static int apply_h_noalloc(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi) {
  if (!c->have_veff) return fail(c, PARO_ERR_STATE, "no effective potential set");
  int st = configure<T>(c);
  if (st) return st;
  const Basis& B = c->bases[ik];
  const int eb = (int)sizeof(cplx<T>);
  const size_t sticks = round256((size_t)nb * c->N[2] * B.ncol * eb);
  const size_t proj = c->have_kb ? round256((size_t)c->nproj * nb * sizeof(double2)) : 0;
  const size_t slice = c->have_kb ? (size_t)c->nproj * nb * sizeof(double2) : 0;  // one split-K slice
  // the FP32 copy of D o P that the FP32 update product reads (the FP64 product reads D o P directly)
  const size_t wconv = c->have_kb && sizeof(T) == 4 ? round256((size_t)c->nproj * nb * sizeof(float2)) : 0;
  const size_t need = sticks + proj + wconv + slice;
  if (need > kNoAllocScratchBytes)
    return fail(c, PARO_ERR_ARG, "paro_apply_h_noalloc: this H psi needs " + std::to_string(need) +
                                     " bytes of scratch, more than the fixed limit of " +
                                     std::to_string(kNoAllocScratchBytes) + " bytes (32 MiB); use fewer bands per call");
  unsigned char* base = nullptr;
  if ((st = noalloc_scratch(c, &base))) return st;
  cplx<T>* S = reinterpret_cast<cplx<T>*>(base);
  const dim3 gz((B.ncol + kStickBatch - 1) / kStickBatch, nb);
  k_zpass_inv<T><<<gz, kZThreads, zpass_smem(c, eb), c->stream>>>(psi, B.npw, S, B.d_col_off, B.d_g_col, B.d_g_z,
                                                                  B.ncol, c->plan[2], tw_of<T>(c, 2), nullptr,
                                                                  kStickBatch);
  PARO_LAUNCH(c, "k_zpass_inv");
  k_plane<T><<<dim3(c->N[2], nb), plane_threads(c), plane_smem(c, eb), c->stream>>>(
      S, B.ncol, B.d_col_x, B.d_col_y, B.d_xrows, B.nxr, c->plan[0], c->plan[1], tw_of<T>(c, 0), tw_of<T>(c, 1),
      vplane_of<T>(c), nullptr);
  PARO_LAUNCH(c, "k_plane");
  k_zpass_fwd<T><<<gz, kZThreads, zpass_smem(c, eb), c->stream>>>(S, psi, B.npw, hpsi, B.npw, kin_of<T>(B), (T)0,
                                                                  B.d_col_off, B.d_g_col, B.d_g_z, B.ncol, c->plan[2],
                                                                  tw_of<T>(c, 2), nullptr, kStickBatch);
  PARO_LAUNCH(c, "k_zpass_fwd");
  if (!c->have_kb) return PARO_OK;
  double2* P = reinterpret_cast<double2*>(base + sticks);
  float2* wf = wconv ? reinterpret_cast<float2*>(base + sticks + proj) : nullptr;
  double2* part = reinterpret_cast<double2*>(base + sticks + proj + wconv);
  const size_t part_elems = (kNoAllocScratchBytes - sticks - proj - wconv) / sizeof(double2);
  if ((st = gemm_cn_scratch<T, T, T>(c, c->nproj, nb, B.npw, beta_of<T>(B), B.npw, psi, B.npw, P, nb, part,
                                     part_elems)))
    return st;
  return gemm_wx<T, T>(c, nb, B.npw, c->nproj, P, nb, false, c->d_dvec, beta_of<T>(B), B.npw, hpsi, B.npw, 1.0, wf);
}

}  // namespace paro

extern "C" int paro_apply_h_noalloc(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, void* hpsi) {
  paro::Ctx* c = paro::unwrap(ctx);
  if (!c) return PARO_ERR_ARG;
  c->err.clear();
  if (ik < 0 || ik >= c->nk || nb < 1 || !psi || !hpsi || psi == hpsi || (dtype != PARO_C64 && dtype != PARO_C32))
    return paro::fail(c, PARO_ERR_ARG, "paro_apply_h_noalloc: bad argument");
  return dtype == PARO_C64 ? paro::apply_h_noalloc<double>(c, ik, nb, static_cast<const double2*>(psi),
                                                           static_cast<double2*>(hpsi))
                           : paro::apply_h_noalloc<float>(c, ik, nb, static_cast<const float2*>(psi),
                                                          static_cast<float2*>(hpsi));
}
