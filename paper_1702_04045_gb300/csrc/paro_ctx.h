// Internal state of a libparo context and the host-side interfaces between its translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/paro.h"
#include "paro_common.cuh"

namespace paro {

// Plane-wave basis of one k-point (Eq. e3) with the z-column ("stick") structure the FFT passes use.
struct Basis {
  int hx_recur = 0;  // ParO iterations of this k-point since H of its Rayleigh-Ritz basis was applied directly
  int npw = 0;
  double kfrac[3] = {0, 0, 0};
  double kcart[3] = {0, 0, 0};
  std::vector<int> miller;        // npw * 3, lexicographic (n1, n2, n3)
  std::vector<double> kin;        // |k+G|^2 / 2
  int ncol = 0;                   // sticks: distinct (n1, n2)
  int nxr = 0;                    // distinct grid rows j1 holding sticks
  int max_run = 0;
  // device
  int* d_miller = nullptr;
  double* d_kin = nullptr;
  float* d_kin32 = nullptr;
  int* d_col_x = nullptr;         // grid row j1 of stick c
  int* d_col_y = nullptr;         // grid column j2 of stick c
  int* d_col_off = nullptr;       // first coefficient of stick c (ncol + 1 entries)
  int* d_g_col = nullptr;         // stick of coefficient g
  int* d_g_z = nullptr;           // grid index j3 of coefficient g
  int* d_xrows = nullptr;         // the nxr rows j1 with sticks
  int* d_xrow_c = nullptr;        // N1 entries: r where d_xrows[r] = j1, or -1 for a row without sticks
  int* d_stick_of = nullptr;      // nxr x N2: the stick at grid row d_xrows[r], column j2, or -1
  int* d_mg = nullptr;            // real-wavefunction mode (k = 0): index of -G for every G
  double2* d_beta = nullptr;      // KB projectors, nproj x npw
  float2* d_beta32 = nullptr;
  // the projectors' TF32 hi/lo split in the shared-memory image of each stage of the tensor-core products
  // (k_tc_beta.cu; formed on first use, dropped when the projectors change)
  float4* d_beta_img_cn = nullptr;
  float4* d_beta_img_wx = nullptr;
  int img_cn_nstage = 0, img_wx_nstage = 0;
  double* d_prec_base = nullptr;  // |k+G|^2/2 (copy used by the preconditioner)
  // orbitals
  double2* d_psi = nullptr;       // n_bands x npw, orthonormal
  double2* d_hpsi = nullptr;      // H psi of the current orbitals
  float2* d_psi32 = nullptr;      // mixed precision: the same orbitals and H psi in FP32
  float2* d_hpsi32 = nullptr;
  // mixed precision: the FP64 orbitals / H psi lag the FP32 ones until a call that reads them (fp64_current)
  bool psi64_stale = false, hpsi64_stale = false;
  bool res_pending = false;       // the residual norms of the last Rayleigh-Ritz step are still in pinned memory
  std::vector<double> eps;        // Ritz values
  std::vector<double> res;        // residual norms
  bool have_psi = false;
};

struct Ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // cell
  double lat[9], bmat[9], omega = 0;
  int nat = 0;
  std::vector<double> pos;
  double ecut = 0;
  int nk = 1;
  std::vector<double> kw;
  int nb = 0, nocc = 0, prec = 0;
  int N[3] = {0, 0, 0};
  int ngrid = 0;
  std::vector<Basis> bases;
  int max_npw = 0;
  FftPlan plan[3];
  double2* d_tw64[3] = {nullptr, nullptr, nullptr};
  float2* d_tw32[3] = {nullptr, nullptr, nullptr};
  // pseudopotentials
  bool have_pp = false;
  double Z = 0, rc = 0, A = 0, a = 0;
  double* d_vloc = nullptr;       // V_loc(r), C order
  bool have_kb = false;
  double kb_rc = 0;
  std::vector<double> D;          // n_atoms * 2
  int nproj = 0;
  double* d_dvec = nullptr;       // D per projector
  float* d_dvec32 = nullptr;
  std::vector<double> beta_norm2_max;  // per (atom, l): max_j ||beta_Ij||^2 over k
  // potential
  bool have_veff = false;
  double* d_veff = nullptr;       // V_eff(r), C order
  double* d_vplane = nullptr;     // V_eff / N_grid, plane-major [z][x][y]
  float* d_vplane32 = nullptr;
  // mean and minimum of V_eff and the PCG shift per k-point: read back from the device without waiting
  // (an event marks the copy); veff_stats() completes the read when a host computation needs them
  double vmean = 0, vmin = 0;
  std::vector<double> sigma_k;
  bool vstats_pending = false;
  double e_ewald = 0;
  // SCF state
  double* d_rho_in = nullptr;
  bool have_rho = false;
  int pulay_n = 0, pulay_head = 0, pulay_cap = 0;
  double* d_pulay_rho = nullptr;  // pulay_cap x ngrid
  double* d_pulay_res = nullptr;
  double* d_pulay_gram = nullptr;  // 16 x 16: <res_s, res_t> by ring slot, filled as residuals arrive
  std::vector<int> pulay_slots;    // host source of the slot list copied each mixing step
  double e_prev = 0;
  int scf_iter = 0, scf_small = 0;
  // occupations: kT = 0, the lowest nocc bands doubly occupied; kT > 0, Fermi-Dirac occupations of the
  // current Ritz values, 2 / (1 + exp((eps - mu)/kT)) with sum_k w_k sum_i f_ik = 2 nocc, and the Mermin
  // free energy E - T S (mts = -T S)
  double kT = 0, mu = 0, mts = 0;
  std::vector<double> occ;  // nk x nb, f_ik
  std::vector<double> occ_key;  // the Ritz values, kT and electron count the occupations were formed from
  int nocc_eff = 0;         // bands per k from the first up to the last with an occupation above 1e-15
  double* d_occ_sqrt = nullptr;  // nk x nb, sqrt(f_ik), for the density of smeared orbitals
  // Gamma-point real-wavefunction mode: the ParO iteration treats its orbitals as real functions (two per
  // packed complex H application and density transform, real Gram and Rayleigh-Ritz matrices);
  // gamma_pack_off suspends it for calls on general complex vectors
  bool gamma_real = false;
  bool gamma_pack_off = false;
  int eig_warm_skip = 0;   // Rayleigh-Ritz eigensolves left before the warm start is tried again
  int eig_warm_fails = 0;  // consecutive warm starts that were not accepted
  float eig_warm_last = 1.f;  // the last correction of the latest warm start (1 before the first)
  unsigned eig_warm_hist = 0;  // the last eight warm starts, bit set when the correction ended below 1e-5
  bool fft_configured[2] = {false, false};
  // instrumentation: kernels launched, and CUDA-event pairs around named kernels while profiling
  long long launches = 0;
  bool prof = false;
  struct ProfEv {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<ProfEv> prof_ev;
  std::vector<cudaEvent_t> prof_pool;  // timing events kept for reuse between recorded ranges
  const char* prof_tag = nullptr;  // phase prefix of recorded names ("pcg", "rr", ...)
  // workspaces by name
  std::map<std::string, std::pair<void*, size_t>> ws;
  // pinned host buffers by name for the small copies of every iteration, each with the event of its last
  // copy: a buffer is rewritten only after that copy has completed, so no copy waits for the stream
  struct Pinned {
    void* h = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
  };
  std::map<std::string, Pinned> pinned;
  int* d_tc_err = nullptr;  // set by a tensor-core kernel whose mbarrier wait gave up
  // FP32 products may run on the tensor cores (3xTF32): inside the inexact inner solves and the adjoint,
  // not in the Rayleigh-Ritz step, the rotations or the energy, which fix the self-consistent result
  bool tc_scope = false;
  struct CholShape {  // launch shape of the cluster Cholesky for order n on device dev
    int n = -1, dev = -1, kind = 0, cls = 0, thr = 0;
    size_t smem = 0;
  } chol_shape;
  std::vector<std::string> chol_pending;  // pinned flags of deferred Cholesky breakdown checks
  bool have_inv_g2 = false;  // the 1/|G|^2 table of the Hartree solve is in the "inv_g2" workspace
  bool have_tw_half = false;  // the N3/2-point FP64 twiddles of the Hartree energy are in "tw64_half"
};

// brings the FP64 orbitals and H psi of a mixed-precision basis up to date with the FP32 ones (api.cu)
int fp64_current(Ctx* c, Basis& b);

// Status helpers (api.cu)
int fail(Ctx* c, int code, const std::string& msg);
int cuda_fail(Ctx* c, cudaError_t e, const char* where);
void* ws_get(Ctx* c, const char* name, size_t bytes);  // nullptr on failure (err set)
// host -> device copy on the context's stream through the pinned buffer `name`; src may change as soon as
// this returns, and the call does not wait for the stream (only, rarely, for the buffer's previous copy)
int h2d_async(Ctx* c, const char* name, void* dst, const void* src, size_t bytes);
// device -> host copy into the pinned buffer `name` (returned in *h) and an event that marks its end;
// the host reads *h after pinned_wait(c, name)
int d2h_async(Ctx* c, const char* name, const void* src, size_t bytes, void** h);
int pinned_wait(Ctx* c, const char* name);
// completes a pending read-back of the V_eff mean and minimum and updates the PCG shifts
int veff_stats(Ctx* c);

#define PARO_CU(c, call)                                               \
  do {                                                                 \
    cudaError_t e__ = (call);                                          \
    if (e__ != cudaSuccess) return ::paro::cuda_fail((c), e__, #call); \
  } while (0)
#define PARO_LAUNCH(c, what)                                                 \
  do {                                                                       \
    cudaError_t e__ = cudaGetLastError();                                    \
    if (e__ != cudaSuccess) return ::paro::cuda_fail((c), e__, what);        \
    ++(c)->launches;                                                         \
  } while (0)

// CUDA events around a named kernel launch on the context's stream (no-ops unless profiling).
cudaEvent_t prof_begin(Ctx* c);
void prof_end(Ctx* c, const char* name, cudaEvent_t a);
// Scoped permission for tensor-core FP32 products (Ctx::tc_scope).
struct TcScope {
  Ctx* c;
  bool old;
  explicit TcScope(Ctx* ctx) : c(ctx), old(ctx->tc_scope) { ctx->tc_scope = true; }
  ~TcScope() { c->tc_scope = old; }
};
// Scoped phase tag: names recorded inside become "tag:name".
struct ProfTag {
  Ctx* c;
  const char* old;
  ProfTag(Ctx* ctx, const char* tag) : c(ctx), old(ctx->prof_tag) { ctx->prof_tag = tag; }
  ~ProfTag() { c->prof_tag = old; }
};

// ---- H psi (k_hpsi.cu) ----
// hpsi = (H - shift) psi for nb bands, T = float or double; active: device int[nb] or nullptr.
// hpsi += dV psi (dV: change of the local potential in the context's V-plane layout and scale); register
// FFT grids only, *used = false otherwise (k_hpsi.cu)
template <typename T>
int apply_dv(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi, const T* dvplane, bool* used);
template <typename T>
int apply_h(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi, double shift, const int* active);
// Checks that the FFT passes support this grid / precision (register and shared-memory budgets).
int check_fft_support(Ctx* c, int elem_bytes);

// ---- dense complex linear algebra (k_linalg.cu) ----
// C[m][n] = sum_k conj(A[m][k]) B[n][k]; A: M x K (lda), B: N x K (ldb); C: M x N (ldc) complex double.
// ACC = double: FP64 throughout. ACC = float: FP32 sums over each K slice, or with carry sums of 16
// consecutive products in FP32 carried into FP64. K-slice partials are summed in double in a fixed order.
// herm: A == B, only tiles with m-tile <= n-tile are computed, the rest mirrored.
template <typename TA, typename TB, typename ACC>
int gemm_cn(Ctx* c, int M, int N, int K, const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb,
            double2* C, int ldc, bool herm, bool carry = false);
// Y[m][n] = beta Y[m][n] + sum_k s_k W(k, m) X[k][n]; W: complex double, element (k, m) at W[k*ldw + m]
// (or at W[m*ldw + k] when wt); s: device double[K] or nullptr (1); X: K x N (ldx) of TX;
// Y: M x N (ldy) of TY; accumulation in TY. wf: device scratch of M K float2 for the FP32 form's converted
// W (nullptr: a workspace of the context, allocated on first use). lower: W(k, m) = 0 for k > m (a
// triangular factor), which lets the FP32 form skip the zero products.
template <typename TX, typename TY>
int gemm_wx(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s, const cplx<TX>* X,
            int ldx, cplx<TY>* Y, int ldy, double beta, float2* wf = nullptr, bool lower = false);
// gemm_cn with the K-slice partials in caller memory (part_elems complex doubles); allocates nothing.
template <typename TA, typename TB, typename ACC>
int gemm_cn_scratch(Ctx* c, int M, int N, int K, const cplx<TA>* A, int lda, const cplx<TB>* B, int ldb,
                    double2* C, int ldc, double2* part, size_t part_elems);
// Tensor-core (tcgen05, 3xTF32) C = conj(A) B^T for gemm_cn<float, float, float> (k_tc.cu); err: time-out flag.
int gemm_cn_tc(Ctx* c, int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, double2* C,
               int ldc, int* err);
// Tensor-core gemm_wx<float, float> (k_tc.cu): Y = beta Y + sum_k s_k W(k, m) X[k].
int gemm_wx_tc(Ctx* c, int M, int N, int K, const double2* W, int ldw, bool wt, const double* s, const float2* X,
               int ldx, float2* Y, int ldy, double beta, int* err);
// Tensor-core paths enabled (not when PARO_NO_TC is set in the environment), and their sticky error flag.
bool tc_enabled();
int* tc_err_flag(Ctx* c);
// enqueues the read-back of the tensor-core error flag (set once a kernel gave up waiting) into pinned
// memory; *h (null when no tensor-core kernel ran) is valid after pinned_wait(c, "tc_err")
int tc_flag_readback(Ctx* c, const int** h);
// ---- tensor-core products with the projectors as the fixed operand (k_tc_beta.cu) ----
int beta_images(Ctx* c, int ik);  // forms the two images of k-point ik if they are missing
// P[p][b] = <beta_p | x_b> for nb rows x (FP32, ld = N_pw)
int gemm_cn_tc_beta(Ctx* c, int ik, int nb, const float2* x, double2* P, int* err);
// y_b += sum_p beta_p D_p P[p][b] (y: nb rows, FP32, ld = N_pw)
int gemm_wx_tc_beta(Ctx* c, int ik, int nb, const double2* P, const double* dvec, float2* y, int* err);
// pieces of k_tc.cu the projector products share
void tc_cn_plan(int M, int N, int K, int* nz_out, int* kslice_out);
int reduce_parts32(Ctx* c, int M, int N, int nz, const float2* part, double2* C, int ldc);
int wx_presplit(Ctx* c, int M, int K, int NT, int KC, const double2* W, int ldw, bool wt, const double* s,
                float4* Wp);
// The context behind a C-ABI handle (api.cu).
Ctx* unwrap(paro_ctx* h);
// Cholesky S = L L^H (n x n, row-major, device), then writes G = conj(L)^{-1} (lower) into g.
// defer: the breakdown flag of the cluster form is read back without waiting, and chol_check() (which waits
// for it) reports a breakdown; the inverse is meaningless until then
// skip (device flag, may be null): when set at run time the cluster Cholesky leaves g as it is and reports
// no breakdown (the factor was formed by orth_first_order); the stream-ordered launch costs no wait.
int chol_inv(Ctx* c, int n, const double2* s, double2* g, bool defer = false, const int* skip = nullptr);
int chol_check(Ctx* c);
// The first-order inverse Cholesky factor of S = I + E when ||E||_F <= tol (decided on the device: *use_dev
// receives the flag for chol_inv's skip).
int orth_first_order(Ctx* c, int n, const double2* s, double2* g, double tol, int** use_dev);
// whether the cluster form of the Cholesky runs for order n on this device (the form that honours skip)
int chol_cluster_available(Ctx* c, int n, bool* avail);
// Hermitian eigensolver, FP64 (k_eigh.cu): w ascending, v columns = eigenvectors (row-major n x n).
int eigh(Ctx* c, int n, const double2* a, double* w, double2* v);
// The same result from an FP32 solve refined in FP64 (k_eigh_mixed.cu); FP64 solver for n > 160. Each
// refinement step squares the eigenvector error across clusters: one step takes the FP32 vectors (~1e-4)
// to ~1e-8 with Rayleigh quotients at FP64 accuracy, two to FP64 vectors.
// warm: the matrix may already be nearly diagonal (a Rayleigh-Ritz basis close to the eigenvectors); then
// two refinement steps from the permutation that sorts its diagonal replace the FP32 solve when their last
// correction is small, with the FP32 solve as the fallback.
// info_out (may be null): instead of waiting for the cluster check, its result is read back into pinned
// memory (*info_out, valid after pinned_wait(c, "eig_info")) and the caller passes it to eigh_mixed_check
// emax_out (may be null): when the last warm starts were well converged, the warm start is not waited for
// either: its last correction is read back into pinned memory (*emax_out, valid after
// pinned_wait(c, "eig_warm_emax")) and the caller passes it to eigh_mixed_accept before using w and v;
// *emax_out is left null when the solve decided by itself
int eigh_mixed(Ctx* c, int n, const double2* a, double* w, double2* v, int refine_steps, bool warm = false,
               const int** info_out = nullptr, const float** emax_out = nullptr);
// the outcome of a deferred warm start from its last correction: true when it is accepted (else the caller solves
// again with warm = false)
bool eigh_mixed_accept(Ctx* c, float emax);
// the end of a mixed solve from its cluster check: the FP64 solver when a cluster could not be resolved
int eigh_mixed_check(Ctx* c, int n, const double2* a, double* w, double2* v, int info);
// Per-band partial sums: out[b] = sum_g Re conj(x[b][g]) y[b][g] (weights optional) — helpers.
template <typename T>
int band_norms(Ctx* c, int nb, int npw, const cplx<T>* x, int ldx, double* out_dev);
// residual norms ||hpsi_b - eps_b psi_b||, eps device
int residual_norms(Ctx* c, int nb, int npw, const double2* psi, const double2* hpsi, const double* eps_dev,
                   double* out_dev);
// the same from FP32 rows in FP32 arithmetic (mixed path)
int residual_norms32(Ctx* c, int nb, int npw, const float2* psi, const float2* hpsi, const double* eps_dev,
                     double* out_dev);
template <typename TS, typename TD>
int convert(Ctx* c, size_t n, const cplx<TS>* src, cplx<TD>* dst);

// ---- KB projectors (k_hpsi.cu) ----
template <typename T>
int kb_apply(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi);

// Suspends the real-wavefunction mode for the scope (calls on general complex vectors, packed rows).
struct GammaPackOff {
  Ctx* c;
  bool old;
  explicit GammaPackOff(Ctx* ctx) : c(ctx), old(ctx->gamma_pack_off) { ctx->gamma_pack_off = true; }
  ~GammaPackOff() { c->gamma_pack_off = old; }
};
inline bool gamma_on(const Ctx* c) { return c->gamma_real && !c->gamma_pack_off; }

// ---- Gamma-point real-wavefunction mode (k_gamma.cu) ----
template <typename T>
int gamma_apply(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* hpsi, double shift, const int* active,
                const T* dvplane, bool* used);
template <typename T>
int gamma_real_rows(Ctx* c, int ik, int nb, cplx<T>* x);   // rows <- their real part, in place
int gamma_real_matrix(Ctx* c, int n, double2* a);          // imaginary parts of an n x n matrix dropped
template <typename T>
int gamma_density_rows(Ctx* c, int ik, int nrow, const cplx<T>* rows, double wfac, double* rho, bool accumulate,
                       int* npacked, const cplx<T>** packed);
int gamma_build_table(Ctx* c, int ik);

// ---- occupations (api.cu) ----
// c->occ, c->nocc_eff, c->mu, c->mts (and d_occ_sqrt with smearing) from the current Ritz values
int update_occupations(Ctx* c);

// ---- setup / SCF (k_scf.cu) ----
int build_vloc(Ctx* c);                   // d_vloc from (Z, rc, A, a)
int build_beta(Ctx* c);                   // d_beta per k
int set_veff_device(Ctx* c, const double* v_dev);  // vplane, sigma, mean
int veff_from_density(Ctx* c, const double* rho_dev, double* eh_out, double* exc_out);
template <typename T>
int density(Ctx* c, const cplx<T>* const* psis, double* rho_dev);  // from given orbitals (occupied)
int energy_terms(Ctx* c, const double* rho_dev, double terms[7]);
int pulay_mix(Ctx* c, const double* rho_out, int depth, double beta);
template <typename T>
int fft3d(Ctx* c, cplx<T>* data, bool inverse);  // in place, unnormalised, C order grid
double ewald(const Ctx* c);

int build_twiddles(Ctx* c);
// radix plan (2, 3, 4, 8) of an FFT of length n (n = 2^a 3^b)
FftPlan fft_plan(int n);
// pass 1 of H psi only (z-inverse FFT of the sticks), FP64, for the density
template <typename T>
int sticks_inverse(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* S);
// density planes with the register FFT (cubic grids it supports); *used = false otherwise
template <typename T>
int density_planes_reg(Ctx* c, int ik, const cplx<T>* S, int nbands, int ngrp, int gsize, double wfac,
                       const double* wsq, double* part, bool* used, bool* f32part);
// rho(r) (+)= wfac sum_b |psi~_b(r)|^2 over nbands rows of psi at k-point ik (psi~: unnormalised inverse DFT)
template <typename T>
// wsq (device, may be null): per-band sqrt(f) of these rows; each band's |psi|^2 is then weighted by f
int density_bands(Ctx* c, int ik, int nbands, const cplx<T>* psi, double wfac, double* rho_dev, bool accumulate,
                  const double* wsq = nullptr);

// ---- adjoint of H psi (k_adjoint.cu, k_scf.cu) ----
int apply_h_adjoint(Ctx* c, int ik, int nb, int dtype, const void* psi, const void* w, void* gpsi, double* gv,
                    double* gpos);
// gpos[I][a] = dL/dR_Ia through V_loc, from gv = dL/dV(r) (device; overwrites gpos)
int vloc_position_grad(Ctx* c, const double* gv, double* gpos);

// ---- batched PCG (k_pcg.cu) ----
template <typename T>
int pcg_run(Ctx* c, int ik, int nb, const cplx<T>* rhs, cplx<T>* x, bool x0_zero, double rel_tol, int max_it,
            int* iters, const cplx<T>* hx0 = nullptr, cplx<T>* hx = nullptr, const cplx<T>* x0src = nullptr,
            const double* fsrc = nullptr);
template <typename T>
int scale_rows(Ctx* c, int nb, int npw, const cplx<T>* x, const double* f_dev, cplx<T>* y);

// ---- batched preconditioned MINRES for the projected correction equations of Algorithm 3 (k_minres.cu) ----
// e_b ~ solution of (I - P_b)(H - eps_b)(I - P_b) e_b = -(H psi_b - eps_b psi_b) on the complement of psi_b;
// eps host double[nb]; iters (host, may be null) receives the steps per orbital.
template <typename T>
int minres_run(Ctx* c, int ik, int nb, const cplx<T>* psi, const cplx<T>* hpsi, const double* eps, cplx<T>* e,
               double rel_tol, int max_it, int* iters);

}  // namespace paro
