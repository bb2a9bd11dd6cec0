// Adjoint (vector-Jacobian product) of H psi. The paper applies H (Eq. e5 with the local
// pseudopotential and Kleinman-Bylander projectors of Section 2.2) but never differentiates it; this
// is the derivative of that operator. For a real loss L of Y = H Psi with cotangent
// W = dL/dRe(Y) + i dL/dIm(Y):
//   dL/dPsi  = H W                                   (H is Hermitian)
//   dL/dV(r) = N^{-1} Re sum_b conj(W~_b(r)) psi~_b(r)   (~: unnormalised inverse DFT on the grid)
//   dL/dR_Ia = local part (V_loc structure factor, k_scf.cu) + KB part:
//              sum_{p in I} D_p sum_b Re[i (conj(A_pb) P^a_pb - conj(A^a_pb) P_pb)],
//              P = beta^H Psi, A = beta^H W, P^a = beta^H (q_a Psi), A^a = beta^H (q_a W), q = k + G.
// dL/dV is formed with the FFT density passes through the polarisation identity
//   4 Re(conj(w) p) = |p + w|^2 - |p - w|^2,
// applied band by band to u_b = c_b (psi_b + s_b W_b), v_b = c_b (psi_b - s_b W_b) with
// s_b = ||psi_b|| / ||W_b|| (so the two terms are of one size and the difference loses no digits to
// an imbalance) and c_b = (4 s_b N)^{-1/2}: then dL/dV = sum_b |u~_b|^2 - |v~_b|^2.
#include "paro_ctx.h"

namespace paro {

template <typename T>
__global__ void k_polarize(int npw, double ngrid, const cplx<T>* __restrict__ psi, const cplx<T>* __restrict__ w,
                           const double* __restrict__ np2, const double* __restrict__ nw2, cplx<T>* __restrict__ u,
                           cplx<T>* __restrict__ v) {
  const int b = blockIdx.y;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npw) return;
  const double a2 = np2[b], b2 = nw2[b];
  const double s = (a2 > 0.0 && b2 > 0.0) ? sqrt(a2 / b2) : 1.0;
  const double cf = 1.0 / sqrt(4.0 * s * ngrid);
  const size_t o = (size_t)b * npw + g;
  const cplx<T> p = psi[o], q = w[o];
  const double px = (double)p.x, py = (double)p.y, qx = s * (double)q.x, qy = s * (double)q.y;
  u[o] = mk<T>((T)(cf * (px + qx)), (T)(cf * (py + qy)));
  v[o] = mk<T>((T)(cf * (px - qx)), (T)(cf * (py - qy)));
}

struct Rec3 {
  double m[9];
};

// Y[b][g] = (k + G_g)_a X[b][g]
template <typename T>
__global__ void k_scale_q(int npw, const int* __restrict__ miller, Rec3 B, double ka, int al,
                          const cplx<T>* __restrict__ X, cplx<T>* __restrict__ Y) {
  const int b = blockIdx.y;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npw) return;
  const double q = ka + miller[3 * g] * B.m[al] + miller[3 * g + 1] * B.m[3 + al] + miller[3 * g + 2] * B.m[6 + al];
  const size_t o = (size_t)b * npw + g;
  const cplx<T> x = X[o];
  Y[o] = mk<T>((T)(q * (double)x.x), (T)(q * (double)x.y));
}

// gpos[I][a] += sum_{p in I} D_p sum_b Re[i (conj(A) P^a - conj(A^a) P)] = -sum D_p sum_b Im(...)
// P, A, Pa[a], Aa[a]: nproj x nb complex (row p, ld nb). One CTA per atom.
__global__ void __launch_bounds__(256) k_kb_force(int nb, const double2* __restrict__ P,
                                                  const double2* __restrict__ A, const double2* __restrict__ Pa,
                                                  const double2* __restrict__ Aa, size_t stride,
                                                  const double* __restrict__ dvec, double* __restrict__ gpos) {
  __shared__ double red[32];
  const int I = blockIdx.x;
  for (int al = 0; al < 3; ++al) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < 4 * nb; t += blockDim.x) {
      const int p = 4 * I + t / nb, b = t % nb;
      const size_t o = (size_t)p * nb + b;
      const double2 a = A[o], pp = P[o], pa = Pa[al * stride + o], aa = Aa[al * stride + o];
      // Im(conj(a) pa - conj(aa) pp)
      const double im = (a.x * pa.y - a.y * pa.x) - (aa.x * pp.y - aa.y * pp.x);
      acc -= dvec[p] * im;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) gpos[3 * I + al] += acc;
  }
}

template <typename T> static const cplx<T>* projectors(const Basis& b);
template <> const double2* projectors<double>(const Basis& b) { return b.d_beta; }
template <> const float2* projectors<float>(const Basis& b) { return b.d_beta32; }

template <typename T>
static int hpsi_adjoint(Ctx* c, int ik, int nb, const cplx<T>* psi, const cplx<T>* w, cplx<T>* gpsi, double* gv,
                        double* gpos) {
  const Basis& B = c->bases[ik];
  const int npw = B.npw;
  const bool f64 = sizeof(T) == 8;
  TcScope tcs(c);  // gradients in FP32 use the 3xTF32 products
  int st;
  if (gpsi && (st = apply_h<T>(c, ik, nb, w, gpsi, 0.0, nullptr))) return st;
  double* gvv = gv;
  if (!gvv && gpos && c->have_pp) {
    gvv = static_cast<double*>(ws_get(c, "adj_gv", (size_t)c->ngrid * sizeof(double)));
    if (!gvv) return PARO_ERR_CUDA;
  }
  if (gvv) {
    double* nrm = static_cast<double*>(ws_get(c, "adj_norms", (size_t)2 * nb * sizeof(double)));
    cplx<T>* u = static_cast<cplx<T>*>(
        ws_get(c, f64 ? "adj_u64" : "adj_u32", (size_t)2 * nb * npw * sizeof(cplx<T>)));
    if (!nrm || !u) return PARO_ERR_CUDA;
    cplx<T>* v = u + (size_t)nb * npw;
    if ((st = band_norms<T>(c, nb, npw, psi, npw, nrm))) return st;
    if ((st = band_norms<T>(c, nb, npw, w, npw, nrm + nb))) return st;
    k_polarize<T><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, (double)c->ngrid, psi, w, nrm, nrm + nb,
                                                                      u, v);
    PARO_LAUNCH(c, "k_polarize");
    if ((st = density_bands<T>(c, ik, nb, u, 1.0, gvv, false))) return st;
    if ((st = density_bands<T>(c, ik, nb, v, -1.0, gvv, true))) return st;
  }
  if (!gpos) return PARO_OK;
  if (c->have_pp) {
    if ((st = vloc_position_grad(c, gvv, gpos))) return st;
  } else {
    PARO_CU(c, cudaMemsetAsync(gpos, 0, (size_t)3 * c->nat * sizeof(double), c->stream));
  }
  if (!c->have_kb || c->nproj == 0) return PARO_OK;
  const int np = c->nproj;
  const size_t mat = (size_t)np * nb;
  double2* M = static_cast<double2*>(ws_get(c, "adj_proj", 8 * mat * sizeof(double2)));
  cplx<T>* Y = static_cast<cplx<T>*>(ws_get(c, f64 ? "adj_y64" : "adj_y32", (size_t)nb * npw * sizeof(cplx<T>)));
  if (!M || !Y) return PARO_ERR_CUDA;
  double2 *P = M, *A = M + mat, *Pa = M + 2 * mat, *Aa = M + 5 * mat;
  const cplx<T>* beta = projectors<T>(B);
  if ((st = gemm_cn<T, T, T>(c, np, nb, npw, beta, npw, psi, npw, P, nb, false, false))) return st;
  if ((st = gemm_cn<T, T, T>(c, np, nb, npw, beta, npw, w, npw, A, nb, false, false))) return st;
  Rec3 R;
  for (int i = 0; i < 9; ++i) R.m[i] = c->bmat[i];
  for (int al = 0; al < 3; ++al) {
    k_scale_q<T><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, B.d_miller, R, B.kcart[al], al, psi, Y);
    PARO_LAUNCH(c, "k_scale_q");
    if ((st = gemm_cn<T, T, T>(c, np, nb, npw, beta, npw, Y, npw, Pa + al * mat, nb, false, false))) return st;
    k_scale_q<T><<<dim3((npw + 255) / 256, nb), 256, 0, c->stream>>>(npw, B.d_miller, R, B.kcart[al], al, w, Y);
    PARO_LAUNCH(c, "k_scale_q");
    if ((st = gemm_cn<T, T, T>(c, np, nb, npw, beta, npw, Y, npw, Aa + al * mat, nb, false, false))) return st;
  }
  k_kb_force<<<c->nat, 256, 0, c->stream>>>(nb, P, A, Pa, Aa, mat, c->d_dvec, gpos);
  PARO_LAUNCH(c, "k_kb_force");
  return PARO_OK;
}

int apply_h_adjoint(Ctx* c, int ik, int nb, int dtype, const void* psi, const void* w, void* gpsi, double* gv,
                    double* gpos) {
  if (dtype == PARO_C64)
    return hpsi_adjoint<double>(c, ik, nb, static_cast<const double2*>(psi), static_cast<const double2*>(w),
                                static_cast<double2*>(gpsi), gv, gpos);
  return hpsi_adjoint<float>(c, ik, nb, static_cast<const float2*>(psi), static_cast<const float2*>(w),
                             static_cast<float2*>(gpsi), gv, gpos);
}

}  // namespace paro
