/*
 * paro.h -- C ABI of libparo, a GB300 (sm_103a) implementation of the data-parallel hot path of the
 * parallel orbital-updating (ParO) plane-wave method for Kohn-Sham DFT (Pan, Dai, de Gironcoli, Gong,
 * Rignanese, Zhou, arXiv:1702.04045).
 *
 * Conventions for every call:
 *   - Hartree atomic units (Section 2.1). A cutoff given in Ry is converted by the caller (1 Ry = 0.5 Ha).
 *   - Every function returns a paro_status (0 = PARO_OK, < 0 = error) and never aborts or exits; the
 *     message of the last error is returned by paro_last_error().
 *   - Complex arrays are interleaved (re, im). Orbital blocks are row-major "band x plane wave": row b
 *     holds the npw coefficients c_{b,k+G} of band b in the basis order reported by paro_miller().
 *   - The caller owns every array argument; the library copies what it keeps. The library owns the
 *     context and all of its device buffers. Device pointers must stay valid for the duration of the
 *     call. All GPU work is enqueued on the context's stream; calls that return host data synchronise.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - There is no CPU fallback: every numerical step runs in this library's CUDA kernels.
 */
#ifndef PARO_H
#define PARO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paro_ctx paro_ctx;

typedef enum {
  PARO_OK = 0,
  PARO_ERR_ARG = -1,           /* bad size, index, pointer or unsupported configuration */
  PARO_ERR_CUDA = -2,          /* a CUDA call failed; the message holds cudaGetErrorString */
  PARO_ERR_BREAKDOWN = -3,     /* PCG p^H A p <= 0 or NaN, or a Cholesky pivot <= 0 */
  PARO_ERR_NOT_CONVERGED = -4, /* SCF / ParO iteration limit reached; the last state is kept */
  PARO_ERR_TIMEOUT = -5,       /* a bounded device-side wait (grid barrier) gave up */
  PARO_ERR_STATE = -6          /* call out of order (e.g. no potential or orbitals set yet) */
} paro_status;

typedef enum { PARO_FP64 = 0, PARO_MIXED = 1 } paro_precision;
typedef enum { PARO_ALG1 = 1, PARO_ALG2 = 2, PARO_ALG3 = 3 } paro_algorithm;
typedef enum { PARO_C64 = 0, PARO_C32 = 1 } paro_dtype; /* complex double / complex float */

/* Energy terms reported by paro_energy / paro_scf (Ha): indices into a double[7]. */
enum {
  PARO_E_KINETIC = 0, PARO_E_NONLOCAL = 1, PARO_E_LOCAL = 2, PARO_E_HARTREE = 3,
  PARO_E_XC = 4, PARO_E_EWALD = 5, PARO_E_TOTAL = 6
};

/*
 * paro_create -- cell, cutoff, k-points and band counts (Section 2.2; Eq. e2, Eq. e3).
 *   lattice   host double[9], rows a1, a2, a3 in Bohr.
 *   pos       host double[n_atoms*3], Cartesian positions in Bohr.
 *   ecut_ha   kinetic cutoff: the basis of k is { G : |k+G|^2/2 <= ecut_ha } (Eq. e3), stored in
 *             lexicographic Miller order (n1, n2, n3).
 *   k_frac    host double[n_k*3], k in reduced coordinates of the reciprocal lattice (NULL: Gamma only,
 *             n_k must be 1); k_w host double[n_k], weights summing to 1 (NULL: 1/n_k each).
 *   n_bands   orbitals per k (occupied + extra); n_occ the occupied ones: 2 n_occ electrons, occupation
 *             2 for each of the lowest n_occ bands, or Fermi-Dirac occupations after paro_set_smearing.
 *   precision PARO_FP64: every step in FP64. PARO_MIXED: orbitals stored in FP32; FFTs, V.psi, the KB
 *             projector products (3xTF32 tensor cores inside the source solves), the inner PCG, the
 *             Cholesky apply and the subspace rotations in FP32; the PCG dot products, the residual
 *             norms and the Gram and H_sub matrices as FP32 partial sums added into an error-free FP32
 *             two-sum pair and returned in FP64; Cholesky factor, Rayleigh-Ritz eigensolve (FP32 solve
 *             refined to FP64 accuracy), density accumulation and energy sums in FP64.
 *   stream    cudaStream_t to enqueue all work on; NULL means the default stream.
 * The FFT grid is the smallest 2^a 3^b per axis with N_i > m_V,i + s_psi,i (m_V: largest |n_i| of the
 * density sphere |G|^2/2 <= 4 ecut; s_psi: span of n_i over every k's basis), so that V.psi is alias
 * free. Errors: PARO_ERR_ARG for non-positive sizes, singular lattice, n_occ > n_bands, n_bands > npw.
 */
int paro_create(paro_ctx** out, const double lattice[9], int n_atoms, const double* pos, double ecut_ha,
                int n_k, const double* k_frac, const double* k_w, int n_bands, int n_occ, int precision,
                void* stream);

/*
 * paro_set_local_pp -- local pseudopotential v(r) = -Z erf(r/rc)/r + A exp(-(r/a)^2) on every atom
 * (Section 2.2, V_loc). V_loc(G) = Omega^{-1} sum_I exp(-i G.R_I) v(G) on the density sphere, with the
 * divergent -4 pi Z/G^2 dropped at G = 0; V_loc(r) by an inverse 3D FFT on the grid. Also sets
 * V_eff = V_loc (a fixed potential) until paro_set_veff / paro_set_density / paro_scf replace it.
 * The ion charge Z also enters the Ewald energy.
 */
int paro_set_local_pp(paro_ctx* ctx, double Z, double rc, double A, double a);

/*
 * paro_set_kb -- Kleinman-Bylander nonlocal part V_nl = sum_{I,j} |beta_Ij> D_{I,l(j)} <beta_Ij|
 * (Section 2.2, V_nl) with four Gaussian projectors per atom (s, px, py, pz), radius rc (Bohr):
 * beta_Ij(k+G) = Omega^{-1/2} exp(-i(k+G).R_I) p~_j(k+G), p~_s = N0 pi^{3/2} rc^3 exp(-q^2 rc^2/4),
 * p~_x = -i N1 (pi^{3/2} rc^5/2) q_x exp(-q^2 rc^2/4), normalised to int p^2 = 1.
 *   D  host double[n_atoms*2]: strength (Ha) of the s and of the p channel of each atom.
 */
int paro_set_kb(paro_ctx* ctx, double rc, const double* D);

/*
 * paro_set_positions -- move the atoms to pos (host double[n_atoms*3], Cartesian Bohr): rebuilds
 * V_loc(r) and the KB projectors from the new structure factors and the Ewald energy; keeps
 * V_eff - V_loc (the Hartree and exchange-correlation part, or whatever part of a set V_eff is not
 * V_loc) and re-takes the Ritz pairs of the current orbitals under the new H.
 */
int paro_set_positions(paro_ctx* ctx, const double* pos);

/* paro_set_veff -- fixed effective potential V_eff(r) (Ha) on the grid, C order (N1, N2, N3);
 * host (on_device = 0) or device (on_device = 1) double[N1*N2*N3]. */
int paro_set_veff(paro_ctx* ctx, const double* v_r, int on_device);
/* paro_set_veff_rest -- V_eff = V_loc(R) + v_rest: the local pseudopotential of the current positions
 * (Section 2.2, V_loc) plus the rest of the effective potential (Hartree, exchange-correlation or any
 * external part; Section 2.1), v_rest host (on_device = 0) or device (on_device = 1) double[N1*N2*N3],
 * C order, Ha. After paro_set_positions this keeps the rest and follows the atoms. PARO_ERR_STATE
 * before paro_set_local_pp. */
int paro_set_veff_rest(paro_ctx* ctx, const double* v_rest, int on_device);
/* paro_get_veff -- copy the current V_eff(r) to a host double[N1*N2*N3]. */
int paro_get_veff(paro_ctx* ctx, double* v_r);
/* paro_get_vloc -- copy the local pseudopotential V_loc(r) of the current positions (Section 2.2,
 * V_loc) to a host double[N1*N2*N3], C order. PARO_ERR_STATE before paro_set_local_pp. */
int paro_get_vloc(paro_ctx* ctx, double* v_r);

/* paro_set_density -- V_eff = V_loc + V_H[rho] + V_xc[rho] from a density rho(r) (electrons/Bohr^3,
 * C order, host or device double[N1*N2*N3]): Hartree V_H(G) = 4 pi rho(G)/G^2 (G != 0), LDA
 * Perdew-Zunger exchange-correlation (Section 2.1, V_H and V_xc). Also becomes the SCF input density. */
int paro_set_density(paro_ctx* ctx, const double* rho, int on_device);

/*
 * paro_set_ecut -- one step of the cutoff ladder of Algorithm 1 (step 2: raise E_cut^(n) to E_cut^(n+1)
 * and go on in the larger plane-wave space V_{N_G^{n+1}}, which contains the old one). The basis of every
 * k-point and the FFT grid are rebuilt for ecut_ha (the rules of paro_create), and with them V_loc and
 * the KB projectors. The orbitals of the old level are embedded in the new basis (new coefficients zero,
 * so they stay orthonormal) and keep their eigenvalue estimates; H psi and the residuals are recomputed.
 * Grid functions are carried to the new grid by Fourier interpolation (their coefficients with
 * |n_i| < N_i/2 on the old grid are kept, exact for band-limited functions): the SCF input density when
 * one is set (V_eff is then rebuilt from it and the Pulay history restarts), else the rest V_eff - V_loc
 * of the set potential. The SCF energy criterion restarts too. ecut_ha below the current cutoff is
 * PARO_ERR_ARG (the same cutoff is a no-op). A batch that holds the context must be destroyed first.
 */
int paro_set_ecut(paro_ctx* ctx, double ecut_ha);

/*
 * paro_set_gamma_real -- the Gamma-point real-wavefunction mode (not in the paper; the standard companion of
 * a plane-wave method at k = 0), for contexts whose only k-point is Gamma. V_eff(r) and the KB projectors
 * are real there, so H maps real orbitals (coefficients with c(-G) = conj(c(G))) to real ones, and the
 * ParO iteration of the context (paro_step, paro_scf_step, paro_scf) then carries two real orbitals in one
 * complex row phi = a + i b: H phi = H a + i H b is split as (H a)(G) = [y(G) + conj(y(-G))]/2,
 * (H b)(G) = [y(G) - conj(y(-G))]/(2i), and |phi(r)|^2 = a(r)^2 + b(r)^2 gives two orbitals' density per
 * transform, which halves the FFT and projector work of H psi and of the density. The Gram and
 * Rayleigh-Ritz matrices are real symmetric (imaginary parts dropped) and orbitals are kept real: orbitals
 * given to paro_set_orbitals / paro_set_state are replaced by their real part (coefficients
 * [c(G) + conj(c(-G))]/2), and enabling the mode does the same to the current orbitals and re-takes their
 * Ritz pairs. Calls on general complex vectors (paro_apply_h, paro_apply_h_adjoint, paro_solve_source,
 * paro_orthonormalize) keep the complex path. enable = 0 leaves the mode. PARO_ERR_ARG for a k-point other
 * than Gamma; batches do not take contexts in this mode.
 */
int paro_set_gamma_real(paro_ctx* ctx, int enable);

/*
 * paro_set_smearing -- occupations of the density and energy (the paper is silent on them; a cell whose
 * highest occupied and lowest empty levels cross has no SCF fixed point at integer occupations).
 * kT = 0 (the default): occupation 2 for the lowest n_occ bands of every k-point. kT > 0 (Ha):
 * Fermi-Dirac occupations of the current Ritz values, f_ik = 2 / (1 + exp((eps_ik - mu)/kT)) over all
 * n_bands, mu fixed by sum_k w_k sum_i f_ik = 2 n_occ, and PARO_E_TOTAL becomes the Mermin free
 * energy E - T S with S = -sum_k w_k sum_i 2 [g ln g + (1 - g) ln(1 - g)], g = f/2. In a ParO-SCF
 * iteration the source solutions carry the occupations of the eigenvalues they were solved with.
 * Errors: PARO_ERR_ARG for a negative or non-finite kT.
 * paro_get_occupations -- the occupations of the current orbitals: f host double[n_k * n_bands] (or
 * NULL), the Fermi level mu (0 without smearing) and the free-energy term -T S (0 without smearing).
 */
int paro_set_smearing(paro_ctx* ctx, double kT);
int paro_get_occupations(paro_ctx* ctx, double* f, double* mu, double* minus_ts);

/* Queries: FFT grid, plane-wave count of k-point ik, Miller indices (host int[npw*3]) of its basis,
 * the PCG shift sigma of the current potential (see paro_solve_source). */
int paro_grid(const paro_ctx* ctx, int n[3]);
int paro_npw(const paro_ctx* ctx, int ik, int* npw);
int paro_miller(const paro_ctx* ctx, int ik, int* hkl);
int paro_sigma(const paro_ctx* ctx, double* sigma);

/*
 * paro_apply_h -- H psi for nb orbitals of k-point ik (Eq. e5, with the potential term read as
 * exp(-i(G_m - G_n).r) and the nonlocal term added):
 *   (H psi)(G) = |k+G|^2/2 c_G + [FFT(V_eff . IFFT(c))](G) / N_grid + sum_p beta_p(G) D_p <beta_p|c>.
 *   dtype  PARO_C64 (complex double) or PARO_C32 (complex float): the arithmetic of the whole apply.
 *   psi    device, nb x npw complex of dtype; hpsi device, same shape (must not alias psi).
 */
int paro_apply_h(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, void* hpsi);

/*
 * paro_apply_vnl -- the nonlocal term of H alone for nb orbitals of k-point ik (Section 2.2's V_nl in the
 * Kleinman-Bylander form):  out_b(G) = sum_p beta_p(G) D_p <beta_p|psi_b>.
 *   dtype  PARO_C64 or PARO_C32, as paro_apply_h; psi, out device, nb x npw complex of dtype (out is
 *          overwritten and must not alias psi).
 *   form   PARO_VNL_ACCURATE: FP64 products (PARO_C64), or FP32 products whose sums are carried in a
 *          two-sum pair (PARO_C32) -- the form the Rayleigh-Ritz step and the energy use;
 *          PARO_VNL_TENSOR (PARO_C32 only): the form of the inexact inner solves, 3xTF32 on the tensor
 *          cores with the projectors' split formed once per position set (relative error about 1e-5).
 *   Errors: PARO_ERR_ARG (bad argument, PARO_VNL_TENSOR with PARO_C64), PARO_ERR_STATE (no projectors
 *   set), PARO_ERR_TIMEOUT (a tensor-core kernel's bounded wait gave up; the output is then undefined).
 */
#define PARO_VNL_ACCURATE 0
#define PARO_VNL_TENSOR 1
int paro_apply_vnl(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, void* out, int form);

/*
 * paro_apply_h_noalloc -- the same H psi as paro_apply_h, for callers that cannot let the library
 * allocate device memory during the call: applications that give all device memory to their own
 * pool up front and run under a fixed budget, and callers that must keep the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree out of a latency-critical loop. The paper has no
 * counterpart; this is a library-interface variant.
 *   Arguments, layout and ownership as paro_apply_h. The call allocates nothing: its scratch (stick
 *   buffer, KB projections, split-K partial sums) is one fixed 32 MiB device array inside the library,
 *   which every GPU that loads the library holds until the process exits.
 *   Size limit: with r(x) = x rounded up to a multiple of 256 bytes, e the bytes of one complex element
 *   of dtype (16 or 8) and P = n_proj * nb, the scratch needed is
 *     r(nb * N3 * (stick columns) * e)                                  (stick buffer)
 *     + [KB projectors only] r(P * 16) + P * 16                          (projections, one K slice)
 *     + [KB projectors and PARO_C32 only] r(P * 8)                       (FP32 copy of D o P)
 *   and must not exceed 32 MiB (33554432 bytes); larger requests fail with PARO_ERR_ARG and a message
 *   giving the bytes needed (split the bands over several calls).
 *   The first call on a device looks up the array's device address (with that device current) and
 *   caches it; make that first call before any stream capture.
 *   Every call shares the one array, and each call overwrites the scratch it reads: calls that
 *   overlap on the GPU (different streams, threads or contexts on the same device) race and must be
 *   serialised by the caller.
 */
int paro_apply_h_noalloc(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, void* hpsi);

/*
 * paro_apply_h_adjoint -- vector-Jacobian product of Y = H Psi (Eq. e5 with V_loc and the KB projectors
 * of Section 2.2). The paper applies H but never differentiates it; this is the derivative of that
 * operator, for gradient-based use of the same Hamiltonian (forces, potential optimisation).
 * For a real loss L with cotangent W = dL/dRe(Y) + i dL/dIm(Y) (so dL = Re sum conj(W) dY):
 *   g_psi = dL/dPsi = H W (same convention);
 *   g_v(r) = dL/dV_eff(r) = N^{-1} Re sum_b conj(W~_b(r)) psi~_b(r), psi~ and W~ the unnormalised
 *            inverse DFTs of the coefficients on the N = N1 N2 N3 grid;
 *   g_pos[I][a] = dL/dR_Ia through the structure factors exp(-i G.R_I) of V_loc (with V_eff - V_loc
 *            held fixed) and exp(-i (k+G).R_I) of the projectors.
 *   psi, w, g_psi: device nb x npw complex of dtype (row = band); g_v: device double[N1*N2*N3]
 *   (C order, overwritten); g_pos: device double[n_atoms*3] (overwritten). g_psi, g_v or g_pos may be
 *   NULL to skip that output. Work runs in the precision of dtype (FP32 FFTs and 3xTF32 tensor-core
 *   projections for PARO_C32), accumulated in FP64. Enqueued on the context stream, no synchronisation.
 */
int paro_apply_h_adjoint(paro_ctx* ctx, int ik, int nb, int dtype, const void* psi, const void* w, void* g_psi,
                         double* g_v, double* g_pos);

/*
 * Batched ParO over many small independent problems -- every k-point of every context in a list,
 * e.g. the k-points of a Monkhorst-Pack mesh or separate cells of uneven size (the paper's two levels
 * of parallelism: orbitals within a problem, problems within the batch). The paper has no batching
 * interface; these calls run Algorithm 1 on all problems at once.
 * paro_batch_create -- groups n_ctx contexts (same precision, same stream, n_bands <= 64 each, a
 *   potential set, not in the real-wavefunction mode). Problems are (context, k-point) pairs in
 *   context-major order. H psi runs as one persistent kernel over flat work lists of all problems'
 *   orbitals (z-FFTs of stick groups, units of one to four z-planes per orbital, z-FFTs back), so a plane
 *   of every problem must fit one CTA's shared memory (N1 x N2 complex elements of the working precision
 *   within 227 KB; otherwise PARO_ERR_ARG). The call times, on the batch's own problems, the unit shapes
 *   (32, 64 or 128 sticks per z-FFT unit; planes per unit for about 2048, 4096 or 8192 points), the launch
 *   forms (one cooperative launch with grid barriers between the phases, or one launch per phase) and the
 *   grids, and keeps the fastest (paro_batch_tuning). The batch refers to the contexts, which must
 *   outlive it.
 * paro_batch_apply_h -- H psi of every problem: psi[i], hpsi[i] device n_bands x npw arrays of dtype
 *   (the contexts' precision: PARO_C64 for FP64, PARO_C32 for mixed) of problem i. Enqueued on the
 *   contexts' stream.
 * paro_batch_step -- one ParO iteration (Algorithm 1, fixed potential) of every problem: source
 *   problems by PCG with a fixed number max_it of steps (each orbital frozen once ||r|| <= rel_tol ||r0||),
 *   Cholesky orthonormalisation, Rayleigh-Ritz with a Jacobi eigensolver per problem, all captured once
 *   into a CUDA graph (re-captured when rel_tol or max_it change) and replayed. The new orbitals,
 *   eigenvalues and residuals are stored in the contexts (paro_get_orbitals etc.); max_resid_out
 *   receives the largest occupied residual. Every context needs orbitals (paro_set_orbitals) first.
 *   Errors: PARO_ERR_BREAKDOWN (PCG or Cholesky), PARO_ERR_NOT_CONVERGED (Jacobi), PARO_ERR_TIMEOUT (a
 *   bounded grid-barrier wait gave up).
 * paro_batch_info -- problems, (problem, band) items, H psi launches per apply (1 or 3), its grid, and
 *   kernels launched per captured step (0 before the first step).
 */
typedef struct paro_batch paro_batch;
int paro_batch_create(paro_batch** out, paro_ctx* const* ctxs, int n_ctx);
int paro_batch_apply_h(paro_batch* b, int dtype, const void* const* psi, void* const* hpsi);
int paro_batch_step(paro_batch* b, double rel_tol, int max_it, double* max_resid_out);
int paro_batch_info(const paro_batch* b, int* n_problems, int* n_items, int* launches_per_apply, int* grid,
                    long long* kernels_per_step);
/* paro_batch_tuning -- the autotuner's measurements at batch creation: n_rows receives the number of
 * candidates timed, and rows (host double[5 * max_rows], may be NULL when max_rows = 0) the first
 * max_rows of them as (launches per H psi: 1 cooperative or 3, grid, sticks per z-FFT unit, plane points
 * per plane unit, ms per H psi of the whole batch). The fastest row is the configuration in use. */
int paro_batch_tuning(const paro_batch* b, int max_rows, int* n_rows, double* rows);
void paro_batch_destroy(paro_batch* b);

/*
 * paro_solve_source -- the independent source problems of Algorithm 1, step 3, for nb orbitals:
 * a(rho; x_i, phi) = (eps_i psi_i, phi), solved shifted as (H - sigma) x_i = (eps_i - sigma) psi_i by
 * batched preconditioned CG started at x_i = psi_i. sigma is a rigorous lower bound of the spectrum
 * minus 0.5 Ha (min V_eff plus the attractive KB channels), so H - sigma is positive definite; the
 * preconditioner is diag(|k+G|^2/2 + mean V_eff - sigma)^{-1}. Each orbital stops once its residual
 * has dropped by rel_tol, or after max_it steps.
 *   eps host double[nb]; psi, x device nb x npw of dtype; iters_out host int[nb] or NULL.
 * Errors: PARO_ERR_BREAKDOWN if p^H A p <= 0 or is not finite for an active orbital.
 */
int paro_solve_source(paro_ctx* ctx, int ik, int nb, int dtype, const double* eps, const void* psi, void* x,
                      double rel_tol, int max_it, int* iters_out);

/*
 * paro_orthonormalize -- the orthonormalisation of Algorithm 1 between the source solutions (step 3)
 * and the Rayleigh-Ritz step (step 4): n rows x_i of k-point ik become orthonormal rows y_i with
 * span{y_1..y_m} = span{x_1..x_m} for every m (Gram-Schmidt in row order, done by Cholesky):
 *   S_ij = <x_i, x_j> = sum_G conj(x_iG) x_jG,  S = L L^H (L lower),  y = conj(L)^{-1} x.
 *   dtype  PARO_C64 (S accumulated in FP64) or PARO_C32 (FP32 rows; S as FP32 sums of 16 products
 *          added into an FP32 two-sum pair); the factorisation and L^{-1} are FP64 for both.
 *   x, y   device n x npw complex of dtype (row = band); y may equal x (in place), else must not overlap.
 * Errors: PARO_ERR_ARG for a bad argument or n > npw; PARO_ERR_BREAKDOWN when a pivot of the
 * factorisation is not positive (rows linearly dependent to working precision).
 */
int paro_orthonormalize(paro_ctx* ctx, int ik, int n, int dtype, const void* x, void* y);

/*
 * paro_set_orbitals -- start vectors of k-point ik (Algorithm 1, step 1): n_bands x npw complex double,
 * host or device. The library orthonormalises them (Cholesky of the Gram matrix, band order) and takes
 * the Ritz pairs of their span under the current potential.
 * paro_get_orbitals -- current orbitals of ik (orthonormal, FP64 complex n_bands x npw), host or device.
 * paro_get_eigenvalues -- current Ritz values, host double[n_k * n_bands], ascending per k.
 * paro_get_residuals -- ||H psi_i - eps_i psi_i||_2 of the current orbitals, host double[n_k * n_bands].
 */
int paro_set_orbitals(paro_ctx* ctx, int ik, const void* psi, int on_device);
int paro_get_orbitals(paro_ctx* ctx, int ik, void* psi, int on_device);
int paro_get_eigenvalues(paro_ctx* ctx, double* eps);
int paro_get_residuals(paro_ctx* ctx, double* res);

/*
 * paro_step -- one ParO iteration at the fixed current potential, for every k-point:
 *   PARO_ALG1 (Algorithm 1): source problems (H - sigma) x_i = (eps_i - sigma) psi_i, Cholesky
 *     orthonormalisation of X, Rayleigh-Ritz in span{x_i}: H_sub = X^H H X, H_sub C = C diag(eps).
 *   PARO_ALG2 (Algorithm 2): corrections (H - sigma) e_i = -(H psi_i - eps_i psi_i) started at e = 0,
 *     projected out of span{psi}; Rayleigh-Ritz in span{psi, e} (dimension up to 2 n_bands).
 *   PARO_ALG3 (Algorithm 3): projected corrections (I - P_i)(H - lambda_i)(I - P_i) e_i = (eps_i - H) psi_i,
 *     P_i = |psi_i><psi_i|, lambda_i (undefined in the paper) read as eps_i; the operator is Hermitian
 *     and indefinite on the complement of psi_i, so each is solved there by preconditioned MINRES from
 *     e = 0 with the projected preconditioner (I - P_i) D (I - P_i), D the PCG preconditioner; then the
 *     Rayleigh-Ritz step of Algorithm 2. rel_tol bounds the MINRES residual estimate's reduction.
 *   rel_tol, max_it: inner PCG stopping rule (see paro_solve_source).
 *   max_resid_out: host, max over k and occupied bands of ||H psi_i - eps_i psi_i|| after the step.
 */
int paro_step(paro_ctx* ctx, int alg, double rel_tol, int max_it, double* max_resid_out);

/*
 * paro_eigh -- Hermitian eigensolver used by the Rayleigh-Ritz step (Algorithm 1 step 4). FP64 contexts:
 * Householder tridiagonalisation, multisection, inverse iteration, back-transformation, all in FP64.
 * Mixed contexts (n <= 160): the same steps in FP32, then two FP64 refinement steps of the eigenvector
 * matrix (Ogita-Aishima) and a Rayleigh-Ritz inside each cluster of close eigenvalues; the result has
 * FP64 accuracy.
 *   a  device n x n complex double, row-major, Hermitian (the lower triangle is read); w device double[n]
 *   ascending eigenvalues; v device n x n complex double, column j = eigenvector j (row-major storage).
 */
int paro_eigh(paro_ctx* ctx, int n, const void* a, double* w, void* v);

/* paro_density -- rho(r) = sum_k w_k sum_i f_ik |psi_ik(r)|^2 of the current orbitals (Section 2.1 and
 * Section 2.2, k-point sum; f_ik = 2 for i < n_occ, or the Fermi-Dirac occupations with smearing),
 * device double[N1*N2*N3], C order. */
int paro_density(paro_ctx* ctx, double* rho_dev);

/* paro_energy -- total energy of the current orbitals and their density (terms as PARO_E_*):
 * sum f <psi|T + V_nl|psi> + int V_loc rho + E_H + E_xc + E_Ewald (point ions, neutralising background);
 * with smearing PARO_E_TOTAL also holds -T S (the Mermin free energy; see paro_get_occupations). */
int paro_energy(paro_ctx* ctx, double terms[7]);

typedef struct {
  int alg;                 /* PARO_ALG1, PARO_ALG2 or PARO_ALG3 */
  double tol_per_atom;     /* stop when |E^{n+1} - E^n| / n_atoms < tol on two consecutive iterations */
  int max_iter;            /* ParO/SCF iterations */
  double inner_rel_tol;    /* PCG residual reduction per source problem */
  int inner_max_it;        /* PCG steps per source problem */
  int pulay_depth;         /* Pulay history length (<= 16) */
  double pulay_beta;       /* Pulay mixing parameter */
} paro_scf_opts;

typedef struct {
  int n_iter;
  int converged;
  double energy[7];
  double max_resid;
} paro_scf_result;

/*
 * paro_scf_step -- one SCF iteration merged with one ParO iteration (Section 2.3, Algorithm 1):
 * V^n from rho_in^n drives the source problems; the density of the Cholesky-orthonormalised solutions
 * is Pulay-mixed into rho_in^{n+1/2}, whose potential drives the Rayleigh-Ritz step; energy terms of
 * the new orbitals are returned (host double[7]). The first call starts from the uniform density.
 * paro_scf -- iterate paro_scf_step until the energy criterion of opts holds (PARO_ERR_NOT_CONVERGED
 * after max_iter, with the last state kept).
 */
int paro_scf_step(paro_ctx* ctx, const paro_scf_opts* opts, double energy[7], double* max_resid_out);
int paro_scf(paro_ctx* ctx, const paro_scf_opts* opts, paro_scf_result* result);

/*
 * paro_set_state -- checkpoint restore: orbitals of k-point ik (n_bands x npw complex double, host or
 * device) and their Ritz values (host double[n_bands]) taken verbatim, no orthonormalisation; H psi
 * and the residual norms are recomputed under the current potential. The caller passes a state saved
 * with paro_get_orbitals / paro_get_eigenvalues (orthonormal orbitals).
 */
int paro_set_state(paro_ctx* ctx, int ik, const void* psi, const double* eps, int on_device);

/*
 * Instrumentation (not part of the method). paro_profile(ctx, 1) starts recording a CUDA event pair
 * on the context's stream around every launch of the named kernels (the three H psi passes, the KB
 * apply, the GEMMs, Cholesky, eigensolver and the PCG vector kernels) and clears earlier records;
 * paro_profile(ctx, 0) stops. paro_profile_read synchronises and returns the number of recorded
 * launches of `name` ("*" for all) and their summed duration in ms; paro_profile_names writes the
 * recorded names, comma separated, into buf[len]. paro_launch_count returns the number of kernels
 * this context has launched since it was created.
 */
int paro_profile(paro_ctx* ctx, int enable);
int paro_profile_read(paro_ctx* ctx, const char* name, int* count, double* total_ms);
int paro_profile_names(paro_ctx* ctx, char* buf, int len);
int paro_launch_count(const paro_ctx* ctx, long long* n);

/* paro_last_error -- message of the last failed call on ctx (or of the last failed paro_create when
 * ctx is NULL); valid until the next call on the same context. */
const char* paro_last_error(const paro_ctx* ctx);

/* paro_destroy -- free the context and all of its device memory (NULL is accepted). */
void paro_destroy(paro_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PARO_H */
