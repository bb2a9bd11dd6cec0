// Cyclic Jacobi eigensolver for a small Hermitian matrix held in shared memory (parallel round-robin
// ordering: n/2 disjoint rotations per round, the column and then the row updates of a round applied by all
// threads). Shared between the batched projection step and the cluster Rayleigh-Ritz of the refinement.
#pragma once

#include "paro_common.cuh"

namespace paro {

// Shared scratch of jacobi_herm: m = n rounded up to even.
struct JacobiScratch {
  int* pos;      // m
  double* rc;    // m / 2
  double* rs;    // m / 2
  double2* rph;  // m / 2
  int* rp;       // m / 2
  int* rq;       // m / 2
  double* red;   // 32
  double* s_off; // 1
  double* s_tot; // 1
};

// A (n x n, leading dimension ldm, shared) is diagonalised in place, V (same layout) accumulates the
// rotations (the caller sets V = I). Stops when the off-diagonal Frobenius norm is below 1e-13 of the whole;
// returns 0 if it is still above 1e-10 of it after 40 sweeps. Every thread of the CTA calls it.
__device__ __forceinline__ int jacobi_herm(int n, int ldm, double2* Am, double2* Vm, JacobiScratch sc) {
#define A(i, j) Am[(i) * ldm + (j)]
#define V(i, j) Vm[(i) * ldm + (j)]
  const int m = n + (n & 1), half = m / 2;
  int* pos = sc.pos;
  double *rc = sc.rc, *rs = sc.rs, *red = sc.red;
  double2* rph = sc.rph;
  int *rp = sc.rp, *rq = sc.rq;
  for (int i = threadIdx.x; i < m; i += blockDim.x) pos[i] = i;
  __syncthreads();
  int converged = 0;
  for (int sweep = 0; sweep < 40 && !converged; ++sweep) {
    for (int round = 0; round < m - 1; ++round) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {  // rotation parameters of this round's pairs
        int p = pos[k], q = pos[m - 1 - k];
        if (p > q) { const int t = p; p = q; q = t; }
        rp[k] = p;
        rq[k] = q;
        rc[k] = 1.0;
        rs[k] = 0.0;
        rph[k] = make_double2(1.0, 0.0);
        if (q < n) {
          const double2 apq = A(p, q);
          const double ab = hypot(apq.x, apq.y);
          if (ab > 0.0) {
            const double tau = (A(q, q).x - A(p, p).x) / (2.0 * ab);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + t * t);
            rc[k] = c;
            rs[k] = t * c;
            rph[k] = make_double2(apq.x / ab, -apq.y / ab);  // exp(-i theta), a_pq = |a_pq| exp(i theta)
          }
        }
      }
      __syncthreads();
      // columns: A <- A U, V <- V U with U_pp = c, U_pq = s, U_qp = -s e^{-i theta}, U_qq = c e^{-i theta}
      for (int t = threadIdx.x; t < half * n; t += blockDim.x) {
        const int k = t / n, i = t % n;
        const int p = rp[k], q = rq[k];
        if (q >= n || rs[k] == 0.0) continue;
        const double c = rc[k], s = rs[k];
        const double2 e = rph[k];
        const double2 ap = A(i, p), aq = A(i, q), vp = V(i, p), vq = V(i, q);
        const double2 eq = cmul(aq, e), ev = cmul(vq, e);
        A(i, p) = make_double2(c * ap.x - s * eq.x, c * ap.y - s * eq.y);
        A(i, q) = make_double2(s * ap.x + c * eq.x, s * ap.y + c * eq.y);
        V(i, p) = make_double2(c * vp.x - s * ev.x, c * vp.y - s * ev.y);
        V(i, q) = make_double2(s * vp.x + c * ev.x, s * vp.y + c * ev.y);
      }
      __syncthreads();
      // rows: A <- U^H A: row p = c A_p - s e^{i theta} A_q, row q = s A_p + c e^{i theta} A_q
      for (int t = threadIdx.x; t < half * n; t += blockDim.x) {
        const int k = t / n, j = t % n;
        const int p = rp[k], q = rq[k];
        if (q >= n || rs[k] == 0.0) continue;
        const double c = rc[k], s = rs[k];
        const double2 ec = cconj(rph[k]);
        const double2 ap = A(p, j), eq = cmul(A(q, j), ec);
        A(p, j) = make_double2(c * ap.x - s * eq.x, c * ap.y - s * eq.y);
        A(q, j) = make_double2(s * ap.x + c * eq.x, s * ap.y + c * eq.y);
      }
      __syncthreads();
      if (threadIdx.x == 0) {  // next round: keep pos[0], rotate the others
        const int last = pos[m - 1];
        for (int i = m - 1; i > 1; --i) pos[i] = pos[i - 1];
        pos[1] = last;
      }
      __syncthreads();
    }
    double off = 0.0, tot = 0.0;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const int r = i / n, c = i % n;
      const double a2 = A(r, c).x * A(r, c).x + A(r, c).y * A(r, c).y;
      tot += a2;
      if (r != c) off += a2;
    }
    off = block_sum(off, red);
    if (threadIdx.x == 0) (*sc.s_off) = off;
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) (*sc.s_tot) = tot;
    __syncthreads();
    converged = (*sc.s_off) <= 1e-26 * (*sc.s_tot) || (*sc.s_off) == 0.0;
  }
  if (!converged && (*sc.s_off) <= 1e-20 * (*sc.s_tot)) converged = 1;  // at the rounding floor
  return converged;
#undef A
#undef V
}

}  // namespace paro
