// Gamma-point real-wavefunction trick (k = 0 only; not in the paper). V_eff(r) and the Kleinman-Bylander
// projectors are real, so H maps real orbitals (coefficients with c(-G) = conj(c(G))) to real orbitals, and
// two of them travel in one complex function phi = a + i b:
//   H phi = H a + i H b, (H a)(G) = [y(G) + conj(y(-G))]/2, (H b)(G) = [y(G) - conj(y(-G))]/(2i), y = H phi;
//   |phi(r)|^2 = a(r)^2 + b(r)^2.
// The ParO iteration of a context in this mode applies H (and the dV term of the Rayleigh-Ritz basis) and
// forms densities on packed pairs: half the FFT and projector work. Its Gram and Rayleigh-Ritz matrices
// are real (imaginary parts dropped) and its orbitals are kept real.
#include "paro_ctx.h"

namespace paro {

// dst[j] = src[2j] + i src[2j+1] (the last row alone when nb is odd)
template <typename T>
__global__ void k_gamma_pack(int npw, int nb, const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst) {
  const int j = blockIdx.y;
  const bool pair = 2 * j + 1 < nb;
  const size_t oa = (size_t)(2 * j) * npw, ob = oa + npw, od = (size_t)j * npw;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
    const cplx<T> a = src[oa + g];
    const cplx<T> b = pair ? src[ob + g] : mk<T>(0, 0);
    dst[od + g] = mk<T>(a.x - b.y, a.y + b.x);
  }
}

// dst[2j] = [y_j(G) + conj(y_j(-G))]/2, dst[2j+1] = -i [y_j(G) - conj(y_j(-G))]/2
template <typename T>
__global__ void k_gamma_unpack(int npw, int nb, const cplx<T>* __restrict__ y, const int* __restrict__ mg,
                               cplx<T>* __restrict__ dst) {
  const int j = blockIdx.y;
  const bool pair = 2 * j + 1 < nb;
  const size_t oy = (size_t)j * npw, oa = (size_t)(2 * j) * npw, ob = oa + npw;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
    const cplx<T> u = y[oy + g], w = y[oy + mg[g]];
    // v = conj(y(-G)); a = (u + v)/2; d = (u - v)/2; b = -i d
    const T vx = w.x, vy = -w.y;
    dst[oa + g] = mk<T>((T)0.5 * (u.x + vx), (T)0.5 * (u.y + vy));
    if (pair) dst[ob + g] = mk<T>((T)0.5 * (u.y - vy), -(T)0.5 * (u.x - vx));
  }
}

// x(G) <- [x(G) + conj(x(-G))]/2 in place; one thread per pair {G, -G} writes both
template <typename T>
__global__ void k_gamma_real(int npw, cplx<T>* __restrict__ x, const int* __restrict__ mg) {
  const size_t o = (size_t)blockIdx.y * npw;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
    const int h = mg[g];
    if (h < g) continue;
    const cplx<T> a = x[o + g], b = x[o + h];
    const cplx<T> r = mk<T>((T)0.5 * (a.x + b.x), (T)0.5 * (a.y - b.y));
    x[o + g] = r;
    x[o + h] = mk<T>(r.x, -r.y);
  }
}

__global__ void k_pair_active(int nb, const int* __restrict__ active, int* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * j >= nb) return;
  out[j] = active[2 * j] || (2 * j + 1 < nb && active[2 * j + 1]) ? 1 : 0;
}

__global__ void k_zero_imag(int n, double2* __restrict__ a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i].y = 0.0;
}

template <typename T>
static cplx<T>* pack_ws(Ctx* c, const char* name, size_t rows, int npw) {
  std::string nm = std::string(name) + (sizeof(T) == 8 ? "64" : "32");
  return static_cast<cplx<T>*>(ws_get(c, nm.c_str(), rows * npw * sizeof(cplx<T>)));
}

template <typename T>
int gamma_pack(Ctx* c, int npw, int nb, const cplx<T>* src, cplx<T>* dst) {
  const int np = (nb + 1) / 2;
  k_gamma_pack<T><<<dim3((npw + 255) / 256, np), 256, 0, c->stream>>>(npw, nb, src, dst);
  PARO_LAUNCH(c, "k_gamma_pack");
  return PARO_OK;
}

template <typename T>
int gamma_real_rows(Ctx* c, int ik, int nb, cplx<T>* x) {
  const Basis& B = c->bases[ik];
  if (!B.d_mg) return fail(c, PARO_ERR_STATE, "real-wavefunction mode without its -G table");
  k_gamma_real<T><<<dim3((B.npw + 255) / 256, nb), 256, 0, c->stream>>>(B.npw, x, B.d_mg);
  PARO_LAUNCH(c, "k_gamma_real");
  return PARO_OK;
}

int gamma_real_matrix(Ctx* c, int n, double2* a) {
  k_zero_imag<<<(n * n + 255) / 256, 256, 0, c->stream>>>(n * n, a);
  PARO_LAUNCH(c, "k_zero_imag");
  return PARO_OK;
}

// (H - shift) psi (dvplane == nullptr) or hpsi += dV psi (dvplane set; *used as apply_dv) of real
// orbitals, two per packed complex row.
template <typename T>
int gamma_apply(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi, double shift, const int* active,
                const T* dvplane, bool* used) {
  const Basis& B = c->bases[ik];
  if (!B.d_mg) return fail(c, PARO_ERR_STATE, "real-wavefunction mode without its -G table");
  const int npw = B.npw, np = (nb + 1) / 2;
  cplx<T>* pin = pack_ws<T>(c, "gamma_in", np, npw);
  cplx<T>* pout = pack_ws<T>(c, "gamma_out", np, npw);
  if (!pin || !pout) return PARO_ERR_CUDA;
  int st = gamma_pack<T>(c, npw, nb, psi, pin);
  if (st) return st;
  int* act2 = nullptr;
  if (active) {
    act2 = static_cast<int*>(ws_get(c, "gamma_active", (size_t)np * sizeof(int)));
    if (!act2) return PARO_ERR_CUDA;
    k_pair_active<<<(np + 127) / 128, 128, 0, c->stream>>>(nb, active, act2);
    PARO_LAUNCH(c, "k_pair_active");
  }
  GammaPackOff off(c);  // the packed rows go through the plain complex path
  if (dvplane) {
    if ((st = gamma_pack<T>(c, npw, nb, hpsi, pout))) return st;
    if ((st = apply_dv<T>(c, ik, np, pin, pout, dvplane, used))) return st;
    if (!*used) return PARO_OK;  // not supported on this grid: the caller applies H instead
  } else if ((st = apply_h<T>(c, ik, np, pin, pout, shift, act2))) {
    return st;
  }
  k_gamma_unpack<T><<<dim3((npw + 255) / 256, np), 256, 0, c->stream>>>(npw, nb, pout, B.d_mg, hpsi);
  PARO_LAUNCH(c, "k_gamma_unpack");
  return PARO_OK;
}

// The density rows (already weighted) packed in pairs: rho(r) (+)= wfac sum_j |a_j + i b_j|^2
template <typename T>
int gamma_density_rows(Ctx* c, int ik, int nrow, const cplx<T>* rows, double wfac, double* rho, bool accumulate,
                       int* npacked, const cplx<T>** packed) {
  const Basis& B = c->bases[ik];
  const int np = (nrow + 1) / 2;
  cplx<T>* p = pack_ws<T>(c, "gamma_dens", np, B.npw);
  if (!p) return PARO_ERR_CUDA;
  int st = gamma_pack<T>(c, B.npw, nrow, rows, p);
  if (st) return st;
  GammaPackOff off(c);
  if ((st = density_bands<T>(c, ik, np, p, wfac, rho, accumulate))) return st;
  *npacked = np;
  *packed = p;
  return PARO_OK;
}

// -G table of the k = 0 basis (host map of the Miller indices); the sphere must be symmetric
int gamma_build_table(Ctx* c, int ik) {
  Basis& B = c->bases[ik];
  std::map<long long, int> where;
  auto key = [](int a, int b, int cc) { return ((long long)(a + 4096) * 8192 + (b + 4096)) * 8192 + (cc + 4096); };
  for (int g = 0; g < B.npw; ++g) where[key(B.miller[3 * g], B.miller[3 * g + 1], B.miller[3 * g + 2])] = g;
  std::vector<int> mg(B.npw);
  for (int g = 0; g < B.npw; ++g) {
    auto it = where.find(key(-B.miller[3 * g], -B.miller[3 * g + 1], -B.miller[3 * g + 2]));
    if (it == where.end()) return fail(c, PARO_ERR_ARG, "real-wavefunction mode: the basis is not symmetric");
    mg[g] = it->second;
  }
  if (!B.d_mg) PARO_CU(c, cudaMalloc(&B.d_mg, (size_t)B.npw * sizeof(int)));
  PARO_CU(c, cudaMemcpyAsync(B.d_mg, mg.data(), mg.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  PARO_CU(c, cudaStreamSynchronize(c->stream));
  return PARO_OK;
}

template int gamma_apply<double>(Ctx*, int, int, const double2*, double2*, double, const int*, const double*, bool*);
template int gamma_apply<float>(Ctx*, int, int, const float2*, float2*, double, const int*, const float*, bool*);
template int gamma_real_rows<double>(Ctx*, int, int, double2*);
template int gamma_real_rows<float>(Ctx*, int, int, float2*);
template int gamma_density_rows<double>(Ctx*, int, int, const double2*, double, double*, bool, int*,
                                        const double2**);
template int gamma_density_rows<float>(Ctx*, int, int, const float2*, double, double*, bool, int*, const float2**);

}  // namespace paro
