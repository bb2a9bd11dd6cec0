// Register-resident line FFTs for the H psi passes.
//
// A line of N = Q * P points is held by a group of P consecutive lanes of a warp, Q values each. In
// the natural layout D_in lane p holds v[q] = x[P q + p]. The unnormalised inverse transform
// (sign +) is the two-factor Cooley-Tukey split n = P q + p, k = k1 + Q k2:
//   A  Q-point DFT over q inside each lane;
//   B  twiddle W_N^{p k1};
//   C  P-point DFT over the lanes by decimation in frequency with warp shuffles, after which lane p
//      holds k2 = bitrev(p): layout D_out, v[k1] = X[k1 + Q bitrev(p)].
// The forward transform (sign -) runs the mirror image, C' (the stages of C in reverse order with the
// decimation-in-time butterfly and conjugate twiddles), B' (W_N^{-k1 p}) and A' (Q-point DFT), and
// maps D_out back to D_in. So an inverse transform, a pointwise product and a forward transform
// need no data movement between lanes beyond the shuffles.
//
// Twiddles come from the table tw[j] = exp(-2 pi i j / N), j < N, in shared memory.
#pragma once

#include "paro_common.cuh"

namespace paro {

template <typename T, bool INV>
__device__ __forceinline__ cplx<T> tw_get(const cplx<T>* tw, int j) {  // exp(-+ 2 pi i j / N)
  const cplx<T> w = tw[j];
  return INV ? cconj(w) : w;
}

template <typename T> __device__ __forceinline__ cplx<T> shfl_xor_c(cplx<T> v, int m) {
  cplx<T> r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return r;
}

template <int P> __device__ __forceinline__ int bitrev_lane(int p) {
  if (P == 1) return 0;
  constexpr int bits = P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;
  return (int)(__brev((unsigned)p) >> (32 - bits));
}

// ---- Q-point DFT in registers, sign by INV; `stride` = N / Q indexes the N-point table ----
template <typename T, int Q, bool INV> struct RegDft;

template <typename T, bool INV> struct RegDft<T, 1, INV> {
  static __device__ __forceinline__ void run(cplx<T>*, const cplx<T>*, int) {}
};
template <typename T, bool INV> struct RegDft<T, 2, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) { dft2<T, INV>(v); }
};
template <typename T, bool INV> struct RegDft<T, 3, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) { dft3<T, INV>(v); }
};
template <typename T, bool INV> struct RegDft<T, 4, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) { dft4<T, INV>(v); }
};
template <typename T, bool INV> struct RegDft<T, 8, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) { dft8<T, INV>(v); }
};

// Q = Q1 Q2: input index q = Q2 q1 + q2, output k = k1 + Q1 k2
template <typename T, int Q1, int Q2, bool INV>
__device__ __forceinline__ void reg_dft_2f(cplx<T>* v, const cplx<T>* tw, int stride) {
  constexpr int Q = Q1 * Q2;
  cplx<T> a[Q];
#pragma unroll
  for (int q2 = 0; q2 < Q2; ++q2) {
    cplx<T> t[Q1];
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) t[q1] = v[Q2 * q1 + q2];
    RegDft<T, Q1, INV>::run(t, tw, stride * Q2);
#pragma unroll
    for (int k1 = 0; k1 < Q1; ++k1)
      a[k1 * Q2 + q2] = (q2 * k1 == 0) ? t[k1] : cmul(t[k1], tw_get<T, INV>(tw, stride * q2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < Q1; ++k1) {
    cplx<T> u[Q2];
#pragma unroll
    for (int q2 = 0; q2 < Q2; ++q2) u[q2] = a[k1 * Q2 + q2];
    RegDft<T, Q2, INV>::run(u, tw, stride * Q1);
#pragma unroll
    for (int k2 = 0; k2 < Q2; ++k2) v[k1 + Q1 * k2] = u[k2];
  }
}

template <typename T, bool INV> struct RegDft<T, 6, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>* tw, int s) { reg_dft_2f<T, 2, 3, INV>(v, tw, s); }
};
// 9 = 3 x 3 as reg_dft_2f<3, 3>, with the twiddles W_9^{q2 k1} (q2 k1 in {1, 2, 4}) as constants
template <typename T, bool INV> struct RegDft<T, 9, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) {
    const T cs[5] = {(T)1, (T)0.766044443118978, (T)0.17364817766693041, (T)0, (T)-0.9396926207859083};
    const T sn[5] = {(T)0, (T)0.6427876096865393, (T)0.984807753012208, (T)0, (T)0.3420201433256689};
    cplx<T> a[9];
#pragma unroll
    for (int q2 = 0; q2 < 3; ++q2) {
      cplx<T> t[3] = {v[q2], v[3 + q2], v[6 + q2]};
      dft3<T, INV>(t);
#pragma unroll
      for (int k1 = 0; k1 < 3; ++k1) {
        const int m = q2 * k1;  // exp(-+ 2 pi i m / 9)
        a[k1 * 3 + q2] = m == 0 ? t[k1] : cmul(t[k1], mk<T>(cs[m], INV ? sn[m] : -sn[m]));
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      cplx<T> u[3] = {a[k1 * 3], a[k1 * 3 + 1], a[k1 * 3 + 2]};
      dft3<T, INV>(u);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) v[k1 + 3 * k2] = u[k2];
    }
  }
};
template <typename T, bool INV> struct RegDft<T, 12, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>* tw, int s) { reg_dft_2f<T, 4, 3, INV>(v, tw, s); }
};
template <typename T, bool INV> struct RegDft<T, 16, INV> {
  static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>* tw, int s) { reg_dft_2f<T, 4, 4, INV>(v, tw, s); }
};

// ---- inverse line transform, D_in -> D_out (sign +, unnormalised) ----
template <typename T, int Q, int P>
__device__ __forceinline__ void line_inv(cplx<T>* v, int p, const cplx<T>* tw) {
  constexpr int N = Q * P;
  RegDft<T, Q, true>::run(v, tw, P);
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1)
    if (p) v[k1] = cmul(v[k1], tw_get<T, true>(tw, p * k1));
#pragma unroll
  for (int h = P / 2; h >= 1; h >>= 1) {
    const bool up = (p & h) != 0;
    const cplx<T> w = tw_get<T, true>(tw, (p & (h - 1)) * (N / (2 * h)));
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const cplx<T> b = shfl_xor_c<T>(v[q], h);
      v[q] = up ? cmul(csub(b, v[q]), w) : cadd(v[q], b);
    }
  }
}

// ---- forward line transform, D_out -> D_in (sign -) ----
template <typename T, int Q, int P>
__device__ __forceinline__ void line_fwd(cplx<T>* v, int p, const cplx<T>* tw) {
  constexpr int N = Q * P;
#pragma unroll
  for (int h = 1; h < P; h <<= 1) {
    const bool up = (p & h) != 0;
    const cplx<T> wc = tw_get<T, false>(tw, (p & (h - 1)) * (N / (2 * h)));
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const cplx<T> t = up ? cmul(v[q], wc) : v[q];
      const cplx<T> o = shfl_xor_c<T>(t, h);
      v[q] = up ? csub(o, t) : cadd(t, o);
    }
  }
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1)
    if (p) v[k1] = cmul(v[k1], tw_get<T, false>(tw, p * k1));
  RegDft<T, Q, false>::run(v, tw, P);
}

// ---- variants with the P-point DFTs of step C done inside the lanes (Q >= P) ----
// Step C needs, for every k1, a P-point DFT over the P lanes of a line. For k1 < P the values go
// through a P x (P + 1) tile in shared memory (row k1 = the P lanes' values of that k1), and lane p
// transforms row k1 = p in registers; the Q - P remaining k1 keep the shuffle stages. One exchange
// through shared memory replaces log2(P) rounds of shuffles for P of the Q values.
// Layout D_T after the inverse: lane p holds v[k2] = X[p + Q k2] (k2 < P) and, for k1 = P + j,
// v[P + j] = X[P + j + Q bitrev(p)]; line_fwd_t maps D_T back to D_in.
// The tile is element e at scr[e * es]: a line's own storage in shared memory (Q P >= P (P + 1)
// elements), free once the line is in registers, or separate memory. ok = false (a lane group without
// a line) skips the tile's stores; its loads must still fall inside shared memory.
template <int Q, int P> __device__ __forceinline__ int dt_index(int p, int pr, int k) {
  return k < P ? p + Q * k : k + Q * pr;
}

// A lane's twiddles of steps B and C for lines of N = Q P, loaded once and kept in registers across the
// lines a warp transforms: b[k1] = W_N^{p k1} (k1 >= 1), c[s] = the shuffle stage h = P / 2^(s+1)'s
// W_N^{(p mod h) N / (2h)} (forward sign; the inverse uses the conjugates).
template <typename T, int Q, int P> struct LaneTw {
  static constexpr int kS = P == 1 ? 1 : (P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5);
  cplx<T> b[Q];
  cplx<T> c[kS];
  __device__ __forceinline__ LaneTw(const cplx<T>* tw, int p) {
    constexpr int N = Q * P;
#pragma unroll
    for (int k1 = 1; k1 < Q; ++k1) b[k1] = tw[p * k1];
    b[0] = mk<T>(1, 0);
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const int h = P >> (s + 1);
      c[s] = h >= 1 ? tw[(p & (h - 1)) * (N / (2 * h))] : mk<T>(1, 0);
    }
  }
};

template <typename T, int Q, int P>
__device__ __forceinline__ void line_inv_t(cplx<T>* v, int p, const cplx<T>* tw, cplx<T>* scr, int es, bool ok) {
  static_assert(Q >= P && Q * P >= P * (P + 1), "line_inv_t needs Q >= P");
  constexpr int N = Q * P;
  __syncwarp();  // every lane has loaded its values before the line's storage is reused
  RegDft<T, Q, true>::run(v, tw, P);
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1)
    if (p) v[k1] = cmul(v[k1], tw_get<T, true>(tw, p * k1));
#pragma unroll
  for (int h = P / 2; h >= 1; h >>= 1) {  // shuffle stages for k1 >= P only
    const bool up = (p & h) != 0;
    const cplx<T> w = tw_get<T, true>(tw, (p & (h - 1)) * (N / (2 * h)));
#pragma unroll
    for (int q = P; q < Q; ++q) {
      const cplx<T> b = shfl_xor_c<T>(v[q], h);
      v[q] = up ? cmul(csub(b, v[q]), w) : cadd(v[q], b);
    }
  }
  if (ok)
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) scr[(k1 * (P + 1) + p) * es] = v[k1];
  __syncwarp();
  cplx<T> u[P];
#pragma unroll
  for (int j = 0; j < P; ++j) u[j] = scr[(p * (P + 1) + j) * es];
  __syncwarp();
  RegDft<T, P, true>::run(u, tw, Q);
#pragma unroll
  for (int k2 = 0; k2 < P; ++k2) v[k2] = u[k2];
}

template <typename T, int Q, int P>
__device__ __forceinline__ void line_fwd_t(cplx<T>* v, int p, const cplx<T>* tw, cplx<T>* scr, int es, bool ok) {
  static_assert(Q >= P && Q * P >= P * (P + 1), "line_fwd_t needs Q >= P");
  constexpr int N = Q * P;
  __syncwarp();  // every lane has loaded its values before the line's storage is reused
  {
    cplx<T> u[P];
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) u[k2] = v[k2];
    RegDft<T, P, false>::run(u, tw, Q);
    if (ok)
#pragma unroll
      for (int j = 0; j < P; ++j) scr[(p * (P + 1) + j) * es] = u[j];
  }
#pragma unroll
  for (int h = 1; h < P; h <<= 1) {  // shuffle stages for k1 >= P only
    const bool up = (p & h) != 0;
    const cplx<T> wc = tw_get<T, false>(tw, (p & (h - 1)) * (N / (2 * h)));
#pragma unroll
    for (int q = P; q < Q; ++q) {
      const cplx<T> t = up ? cmul(v[q], wc) : v[q];
      const cplx<T> o = shfl_xor_c<T>(t, h);
      v[q] = up ? csub(o, t) : cadd(t, o);
    }
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) v[k1] = scr[(k1 * (P + 1) + p) * es];
  __syncwarp();
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1)
    if (p) v[k1] = cmul(v[k1], tw_get<T, false>(tw, p * k1));
  RegDft<T, Q, false>::run(v, tw, P);
}

// line_inv_t / line_fwd_t with the lane's twiddles from registers (lt) instead of the table
template <typename T, int Q, int P>
__device__ __forceinline__ void line_inv_tr(cplx<T>* v, int p, const LaneTw<T, Q, P>& lt, cplx<T>* scr, int es,
                                            bool ok) {
  static_assert(Q == 9 && P <= 8, "line_inv_tr: constant-twiddle Q-point DFT (Q = 9) only");
  __syncwarp();  // every lane has loaded its values before the line's storage is reused
  RegDft<T, Q, true>::run(v, nullptr, P);
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1)
    if (p) v[k1] = cmul(v[k1], cconj(lt.b[k1]));
#pragma unroll
  for (int s = 0; (P >> (s + 1)) >= 1; ++s) {  // shuffle stages h = P/2 .. 1 for k1 >= P only
    const int h = P >> (s + 1);
    const bool up = (p & h) != 0;
    const cplx<T> w = cconj(lt.c[s]);
#pragma unroll
    for (int q = P; q < Q; ++q) {
      const cplx<T> b = shfl_xor_c<T>(v[q], h);
      v[q] = up ? (h > 1 ? cmul(csub(b, v[q]), w) : csub(b, v[q])) : cadd(v[q], b);
    }
  }
  if (ok)
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) scr[(k1 * (P + 1) + p) * es] = v[k1];
  __syncwarp();
  cplx<T> u[P];
#pragma unroll
  for (int j = 0; j < P; ++j) u[j] = scr[(p * (P + 1) + j) * es];
  __syncwarp();
  RegDft<T, P, true>::run(u, nullptr, Q);
#pragma unroll
  for (int k2 = 0; k2 < P; ++k2) v[k2] = u[k2];
}

template <typename T, int Q, int P>
__device__ __forceinline__ void line_fwd_tr(cplx<T>* v, int p, const LaneTw<T, Q, P>& lt, cplx<T>* scr, int es,
                                            bool ok) {
  static_assert(Q == 9 && P <= 8, "line_fwd_tr: constant-twiddle Q-point DFT (Q = 9) only");
  __syncwarp();  // every lane has loaded its values before the line's storage is reused
  {
    cplx<T> u[P];
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) u[k2] = v[k2];
    RegDft<T, P, false>::run(u, nullptr, Q);
    if (ok)
#pragma unroll
      for (int j = 0; j < P; ++j) scr[(p * (P + 1) + j) * es] = u[j];
  }
#pragma unroll
  for (int s = LaneTw<T, Q, P>::kS - 1; s >= 0; --s) {  // shuffle stages h = 1 .. P/2 for k1 >= P only
    const int h = P >> (s + 1);
    if (h < 1) continue;
    const bool up = (p & h) != 0;
    const cplx<T> wc = lt.c[s];
#pragma unroll
    for (int q = P; q < Q; ++q) {
      const cplx<T> t = up && h > 1 ? cmul(v[q], wc) : v[q];
      const cplx<T> o = shfl_xor_c<T>(t, h);
      v[q] = up ? csub(o, t) : cadd(t, o);
    }
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) v[k1] = scr[(k1 * (P + 1) + p) * es];
  __syncwarp();
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1)
    if (p) v[k1] = cmul(v[k1], lt.b[k1]);
  RegDft<T, Q, false>::run(v, nullptr, P);
}

// Factorisations N = Q * P used by the register kernels (P lanes per line, Q values per lane).
template <int N> struct LineShape;
template <> struct LineShape<32> { static constexpr int Q = 4, P = 8; };
template <> struct LineShape<36> { static constexpr int Q = 9, P = 4; };
template <> struct LineShape<48> { static constexpr int Q = 6, P = 8; };
template <> struct LineShape<72> { static constexpr int Q = 9, P = 8; };
template <> struct LineShape<128> { static constexpr int Q = 8, P = 16; };

}  // namespace paro
