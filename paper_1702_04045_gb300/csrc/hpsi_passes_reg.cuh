// Register-FFT H psi passes; included by k_hpsi.cu after its helpers (kStickBatch, tw_of, vplane_of,
// kin_of), inside namespace paro.
#pragma once

// ------------------------------------------------------------------------------------------------
// Register-FFT versions of the three passes for cubic grids N^3 with N in {32, 36, 48, 72, 128}
// (line FFTs of fft_reg.cuh: one group of P lanes per line, Q values per lane).
// ------------------------------------------------------------------------------------------------
// FP32 lines with Q > P keep step C in the lanes (line_inv_t / line_fwd_t). The z-passes and the density
// pass exchange through the line's own storage in shared memory; the plane pass, whose column tiles
// would meet two-way bank conflicts in both directions, gives each lane group of a warp its own tile
// (kWarpTile elements per warp).
template <typename T, int N> struct PlaneLines {
  static constexpr int Q = LineShape<N>::Q, P = LineShape<N>::P;
  static constexpr bool kTile = sizeof(T) == 4 && Q > P;
  static constexpr int kWarpTile = kTile ? (32 / P) * P * (P + 1) : 0;
};

template <typename T, int N3>
__global__ void __launch_bounds__(256) k_zpass_inv_reg(const cplx<T>* __restrict__ psi, int ldpsi,
                                                       cplx<T>* __restrict__ S, const int* __restrict__ col_off,
                                                       const int* __restrict__ g_col, const int* __restrict__ g_z,
                                                       int ncol, const cplx<T>* __restrict__ twz,
                                                       const int* __restrict__ active, int CB) {
  using SH = LineShape<N3>;
  constexpr int Q = SH::Q, P = SH::P, LS = N3 + 1, G = 32 / P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* line = tw + N3;
  const int b = blockIdx.y;
  if (active != nullptr && active[b] == 0) return;
  const int c0 = blockIdx.x * CB;
  const int ncb = min(CB, ncol - c0);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) tw[i] = twz[i];
  for (int i = threadIdx.x; i < ncb * LS; i += blockDim.x) line[i] = mk<T>(0, 0);
  __syncthreads();
  const int g0 = col_off[c0], g1 = col_off[c0 + ncb];
  const cplx<T>* pp = psi + (size_t)b * ldpsi;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) line[(g_col[g] - c0) * LS + g_z[g]] = pp[g];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
  for (int l0 = warp * G; l0 < ncb; l0 += nw * G) {
    const int l = l0 + grp;
    const bool ok = l < ncb;
    cplx<T>* ln = line + (ok ? l : 0) * LS;
    cplx<T> v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = ok ? ln[P * q + p] : mk<T>(0, 0);
    if constexpr (PlaneLines<T, N3>::kTile) line_inv_t<T, Q, P>(v, p, tw, ln, 1, ok);
    else line_inv<T, Q, P>(v, p, tw);
    __syncwarp();
    if (ok)
#pragma unroll
      for (int k = 0; k < Q; ++k) ln[PlaneLines<T, N3>::kTile ? dt_index<Q, P>(p, pr, k) : k + Q * pr] = v[k];
    __syncwarp();
  }
  __syncthreads();
  cplx<T>* Sb = S + (size_t)b * N3 * ncol;
  for (int i = threadIdx.x; i < N3 * ncb; i += blockDim.x) {
    const int z = i / ncb, cc = i - z * ncb;
    Sb[(size_t)z * ncol + c0 + cc] = line[cc * LS + z];
  }
}

// Warps per plane-pass CTA: 9 for N = 72 (a warp holds 4 lines of 8 lanes, so the ~35 stick rows of the
// y-pass take one round of 36 lines and the 72 columns of the x-pass two), 8 otherwise.
template <int N> struct PlaneWarps { static constexpr int value = 8; };
template <> struct PlaneWarps<72> { static constexpr int value = 9; };
// Row stride of the plane in shared memory (complex elements). The x-pass reads a column with 8 lanes
// per line and 4 lines per warp: with a stride of 74 (10 mod 16) the 16 8-byte elements of a half-warp fall
// in distinct bank pairs, where 73 gave two-way conflicts.
template <int N> struct PlaneStride { static constexpr int value = N + 1; };
template <> struct PlaneStride<72> { static constexpr int value = 74; };

// Resident CTAs per SM the plane pass is compiled for (a register cap of 65536 / (CTAs x threads)): the
// compact FP32 plane of the 72-point grid lets four CTAs of nine warps share an SM.
template <typename T, int N> struct PlaneMinBlocks { static constexpr int value = 1; };
template <> struct PlaneMinBlocks<float, 72> { static constexpr int value = 4; };

// Shared memory of the plane pass: the warps' exchange tiles, the row-offset table and the nxr stick rows
// of the plane.
template <typename T, int N>
static size_t plane_reg_smem(int nxr) {
  constexpr int kWT = PlaneLines<T, N>::kWarpTile;
  return sizeof(cplx<T>) * (PlaneWarps<N>::value * kWT + (size_t)nxr * PlaneStride<N>::value) + N * sizeof(int);
}

// The plane is kept compact in shared memory: only its nxr rows that hold sticks (row r at Pl + r LS is
// grid row xrows[r]; xrow_c maps a grid row to r or -1). The inverse pass along y reads its lines straight
// from the stick buffer (stick_of[r N2 + j2]: the stick at grid row xrows[r], column j2, or -1) and the
// forward pass writes them straight back, so the plane is neither cleared nor scattered nor gathered. The
// inverse transform along x reads the rows without sticks as the zeros they are, and the forward transform
// writes back only the stick rows, which are all that the forward pass along y reads. Two block barriers
// per plane; the twiddles are read through the L1 cache.
template <typename T, int N1, int N2, int NW = PlaneWarps<N1>::value>
__global__ void __launch_bounds__(32 * NW, PlaneMinBlocks<T, N1>::value)
    k_plane_reg(cplx<T>* __restrict__ S, int ncol, const int* __restrict__ stick_of, const int* __restrict__ xrow_c,
                int nxr, const cplx<T>* __restrict__ twx, const cplx<T>* __restrict__ twy,
                const T* __restrict__ vplane, const int* __restrict__ active) {
  using SX = LineShape<N1>;
  using SY = LineShape<N2>;
  using LX = PlaneLines<T, N1>;
  using LY = PlaneLines<T, N2>;
  constexpr int LS = PlaneStride<N2>::value;
  static_assert(N1 % 4 == 0, "row-offset table keeps the plane 16-byte aligned");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tiles = reinterpret_cast<cplx<T>*>(smem_raw);  // per warp: the larger of the two lines' kWarpTile
  constexpr int kWT = LX::kWarpTile > LY::kWarpTile ? LX::kWarpTile : LY::kWarpTile;
  int* roff = reinterpret_cast<int*>(tiles + NW * kWT);  // grid row -> offset of its compact row, or -1
  cplx<T>* Pl = reinterpret_cast<cplx<T>*>(roff + N1);
  const int z = blockIdx.x, b = blockIdx.y, N3 = gridDim.x;
  if (active != nullptr && active[b] == 0) return;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) {
    const int r = xrow_c[i];
    roff[i] = r >= 0 ? r * LS : -1;
  }
  cplx<T>* Sz = S + ((size_t)b * N3 + z) * ncol;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  {  // inverse along y, rows that hold sticks, from the stick buffer
    constexpr int Q = SY::Q, P = SY::P, G = 32 / P;
    const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
    for (int r0 = warp * G; r0 < nxr; r0 += nw * G) {
      const int r = r0 + grp;
      const bool ok = r < nxr;
      const int* so = stick_of + (size_t)(ok ? r : 0) * N2;
      cplx<T> v[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int cs = ok ? so[P * q + p] : -1;
        v[q] = cs >= 0 ? Sz[cs] : mk<T>(0, 0);
      }
      if constexpr (LY::kTile) line_inv_t<T, Q, P>(v, p, twy, tiles + warp * kWT + grp * P * (P + 1), 1, true);
      else line_inv<T, Q, P>(v, p, twy);
      if (ok) {
        cplx<T>* row = Pl + r * LS;
#pragma unroll
        for (int k = 0; k < Q; ++k) row[LY::kTile ? dt_index<Q, P>(p, pr, k) : k + Q * pr] = v[k];
      }
    }
  }
  __syncthreads();
  {  // along x for every column: inverse, times V / N_grid, forward (all in registers)
    constexpr int Q = SX::Q, P = SX::P, G = 32 / P;
    const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
    const T* V = vplane + (size_t)z * N1 * N2;
    for (int c0 = warp * G; c0 < N2; c0 += nw * G) {
      const int y = c0 + grp;
      const bool ok = y < N2;
      cplx<T> v[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int o = roff[P * q + p];
        v[q] = ok && o >= 0 ? Pl[o + y] : mk<T>(0, 0);
      }
      if constexpr (LX::kTile) {
        cplx<T>* tile = tiles + warp * kWT + grp * P * (P + 1);
        line_inv_t<T, Q, P>(v, p, twx, tile, 1, true);
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = cscale(v[k], ok ? V[dt_index<Q, P>(p, pr, k) * N2 + y] : (T)0);
        line_fwd_t<T, Q, P>(v, p, twx, tile, 1, true);
      } else {
        line_inv<T, Q, P>(v, p, twx);
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = cscale(v[k], ok ? V[(k + Q * pr) * N2 + y] : (T)0);
        line_fwd<T, Q, P>(v, p, twx);
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int o = roff[P * q + p];
        if (ok && o >= 0) Pl[o + y] = v[q];
      }
    }
  }
  __syncthreads();
  {  // forward along y, rows that hold sticks, into the stick buffer
    constexpr int Q = SY::Q, P = SY::P, G = 32 / P;
    const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
    for (int r0 = warp * G; r0 < nxr; r0 += nw * G) {
      const int r = r0 + grp;
      const bool ok = r < nxr;
      const cplx<T>* row = Pl + (ok ? r : 0) * LS;
      cplx<T> v[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) v[k] = ok ? row[LY::kTile ? dt_index<Q, P>(p, pr, k) : k + Q * pr] : mk<T>(0, 0);
      if constexpr (LY::kTile) line_fwd_t<T, Q, P>(v, p, twy, tiles + warp * kWT + grp * P * (P + 1), 1, true);
      else line_fwd<T, Q, P>(v, p, twy);
      if (ok) {
        const int* so = stick_of + (size_t)r * N2;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int cs = so[P * q + p];
          if (cs >= 0) Sz[cs] = v[q];
        }
      }
    }
  }
}

// ACC: hpsi += the transformed potential term alone (no kinetic or shift term)
template <typename T, int N3, bool ACC = false>
__global__ void __launch_bounds__(256) k_zpass_fwd_reg(const cplx<T>* __restrict__ S, const cplx<T>* __restrict__ psi,
                                                       int ldpsi, cplx<T>* __restrict__ hpsi, int ldh,
                                                       const T* __restrict__ kin, T shift,
                                                       const int* __restrict__ col_off, const int* __restrict__ g_col,
                                                       const int* __restrict__ g_z, int ncol,
                                                       const cplx<T>* __restrict__ twz,
                                                       const int* __restrict__ active, int CB) {
  using SH = LineShape<N3>;
  constexpr int Q = SH::Q, P = SH::P, LS = N3 + 1, G = 32 / P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* line = tw + N3;
  const int b = blockIdx.y;
  if (active != nullptr && active[b] == 0) return;
  const int c0 = blockIdx.x * CB;
  const int ncb = min(CB, ncol - c0);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) tw[i] = twz[i];
  const cplx<T>* Sb = S + (size_t)b * N3 * ncol;
  for (int i = threadIdx.x; i < N3 * ncb; i += blockDim.x) {
    const int z = i / ncb, cc = i - z * ncb;
    line[cc * LS + z] = Sb[(size_t)z * ncol + c0 + cc];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
  for (int l0 = warp * G; l0 < ncb; l0 += nw * G) {
    const int l = l0 + grp;
    const bool ok = l < ncb;
    cplx<T>* ln = line + (ok ? l : 0) * LS;
    cplx<T> v[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) v[k] = ok ? ln[PlaneLines<T, N3>::kTile ? dt_index<Q, P>(p, pr, k) : k + Q * pr] : mk<T>(0, 0);
    if constexpr (PlaneLines<T, N3>::kTile) line_fwd_t<T, Q, P>(v, p, tw, ln, 1, ok);
    else line_fwd<T, Q, P>(v, p, tw);
    __syncwarp();
    if (ok)
#pragma unroll
      for (int q = 0; q < Q; ++q) ln[P * q + p] = v[q];
    __syncwarp();
  }
  __syncthreads();
  const int g0 = col_off[c0], g1 = col_off[c0 + ncb];
  const cplx<T>* pp = psi + (size_t)b * ldpsi;
  cplx<T>* h = hpsi + (size_t)b * ldh;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const cplx<T> v = line[(g_col[g] - c0) * LS + g_z[g]];
    if (ACC) {
      h[g] = cadd(h[g], v);
    } else {
      const cplx<T> cc = pp[g];
      const T t = kin[g] - shift;
      h[g] = mk<T>(v.x + t * cc.x, v.y + t * cc.y);
    }
  }
}

// dynamic shared memory limit, set once per kernel instantiation and device
template <typename K> static int set_smem_once(Ctx* c, K kernel, int* done) {
  int dev = 0;
  PARO_CU(c, cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && done[dev]) return PARO_OK;
  PARO_CU(c, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  PARO_CU(c, cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  if (dev >= 0 && dev < 64) done[dev] = 1;
  return PARO_OK;
}

template <typename T, int N>
static int passes_reg(Ctx* c, const Basis& B, int nb, const cplx<T>* psi, cplx<T>* S, cplx<T>* hpsi, double shift,
                      const int* active, const T* vplane = nullptr, bool acc = false) {
  static int done[4][64];
  const int eb = (int)sizeof(cplx<T>);
  const bool f64 = sizeof(T) == 8;
  const size_t smz = (size_t)eb * (N + kStickBatch * (N + 1));
  constexpr int kPW = PlaneWarps<N>::value;
  const size_t smp = plane_reg_smem<T, N>(B.nxr);
  int st;
  if ((st = set_smem_once(c, k_zpass_inv_reg<T, N>, done[0])) || (st = set_smem_once(c, k_plane_reg<T, N, N>, done[1])) ||
      (st = set_smem_once(c, k_zpass_fwd_reg<T, N>, done[2])) ||
      (st = set_smem_once(c, k_zpass_fwd_reg<T, N, true>, done[3])))
    return st;
  const dim3 gz((B.ncol + kStickBatch - 1) / kStickBatch, nb);
  cudaEvent_t ev = prof_begin(c);
  k_zpass_inv_reg<T, N><<<gz, 256, smz, c->stream>>>(psi, B.npw, S, B.d_col_off, B.d_g_col, B.d_g_z, B.ncol,
                                                     tw_of<T>(c, 2), active, kStickBatch);
  PARO_LAUNCH(c, "k_zpass_inv_reg");
  prof_end(c, f64 ? "k_zpass_inv<f64>" : "k_zpass_inv<f32>", ev);
  ev = prof_begin(c);
  k_plane_reg<T, N, N><<<dim3(c->N[2], nb), 32 * kPW, smp, c->stream>>>(S, B.ncol, B.d_stick_of, B.d_xrow_c, B.nxr,
                                                                   tw_of<T>(c, 0), tw_of<T>(c, 1),
                                                                   vplane ? vplane : vplane_of<T>(c), active);
  PARO_LAUNCH(c, "k_plane_reg");
  prof_end(c, f64 ? "k_plane<f64>" : "k_plane<f32>", ev);
  ev = prof_begin(c);
  if (acc)
    k_zpass_fwd_reg<T, N, true><<<gz, 256, smz, c->stream>>>(S, psi, B.npw, hpsi, B.npw, kin_of<T>(B), (T)shift,
                                                             B.d_col_off, B.d_g_col, B.d_g_z, B.ncol, tw_of<T>(c, 2),
                                                             active, kStickBatch);
  else
    k_zpass_fwd_reg<T, N><<<gz, 256, smz, c->stream>>>(S, psi, B.npw, hpsi, B.npw, kin_of<T>(B), (T)shift,
                                                       B.d_col_off, B.d_g_col, B.d_g_z, B.ncol, tw_of<T>(c, 2), active,
                                                       kStickBatch);
  PARO_LAUNCH(c, "k_zpass_fwd_reg");
  prof_end(c, f64 ? "k_zpass_fwd<f64>" : "k_zpass_fwd<f32>", ev);
  return PARO_OK;
}

// Register kernels when the grid is N^3 with a supported N and the plane fits in shared memory.
template <typename T>
static int passes_reg_dispatch(Ctx* c, const Basis& B, int nb, const cplx<T>* psi, cplx<T>* S, cplx<T>* hpsi,
                               double shift, const int* active, bool* used, const T* vplane = nullptr,
                               bool acc = false) {
  *used = false;
  const int n = c->N[0];
  if (c->N[1] != n || c->N[2] != n) return PARO_OK;
  if ((size_t)sizeof(cplx<T>) * (2 * n + n * (n + (n == 72 ? 2 : 1))) > 227 * 1024) return PARO_OK;  // PlaneStride
  *used = true;
  switch (n) {
    case 32: return passes_reg<T, 32>(c, B, nb, psi, S, hpsi, shift, active, vplane, acc);
    case 36: return passes_reg<T, 36>(c, B, nb, psi, S, hpsi, shift, active, vplane, acc);
    case 48: return passes_reg<T, 48>(c, B, nb, psi, S, hpsi, shift, active, vplane, acc);
    case 72: return passes_reg<T, 72>(c, B, nb, psi, S, hpsi, shift, active, vplane, acc);
    case 128: return passes_reg<T, 128>(c, B, nb, psi, S, hpsi, shift, active, vplane, acc);
    default: *used = false; return PARO_OK;
  }
}

// Density planes with the register FFT: per (z-plane, band group) the inverse transforms along y and
// x of each band, |psi(r)|^2 summed in shared memory, the group's plane written to part.
// TACC: accumulator of the |psi|^2 sum over the group's bands (at most gsize = 8): float for FP32 orbitals
// (an 8-term FP32 sum, the groups then summed in FP64 by the caller), double for FP64 orbitals.
// The plane is compact as in k_plane_reg (stick rows only, lines along y read straight from the stick
// buffer); two block barriers per band.
template <typename T, int N1, int N2, typename TACC, int NW = PlaneWarps<N1>::value>
__global__ void __launch_bounds__(32 * NW) k_plane_density_reg(const cplx<T>* __restrict__ S, int ncol, int nbands,
                                                           int gsize, const int* __restrict__ stick_of,
                                                           const int* __restrict__ xrow_c, int nxr,
                                                           const cplx<T>* __restrict__ twx,
                                                           const cplx<T>* __restrict__ twy, double wfac,
                                                           const double* __restrict__ wsq,
                                                           double* __restrict__ part) {
  using SX = LineShape<N1>;
  using SY = LineShape<N2>;
  using LX = PlaneLines<T, N1>;
  using LY = PlaneLines<T, N2>;
  constexpr int LS = PlaneStride<N2>::value;
  constexpr int kWT = LX::kWarpTile > LY::kWarpTile ? LX::kWarpTile : LY::kWarpTile;
  static_assert(N1 % 4 == 0, "row-offset table keeps the plane 16-byte aligned");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TACC* acc = reinterpret_cast<TACC*>(smem_raw);  // N1 N2, a multiple of 16 bytes
  cplx<T>* tx = reinterpret_cast<cplx<T>*>(acc + N1 * N2);  // twiddles in shared memory: the lanes' register
  cplx<T>* ty = tx + N1;                                    // copies are formed again for every band
  cplx<T>* tiles = ty + N2;
  int* roff = reinterpret_cast<int*>(tiles + NW * kWT);
  cplx<T>* Pl = reinterpret_cast<cplx<T>*>(roff + N1);
  const int z = blockIdx.x, grp_b = blockIdx.y, N3 = gridDim.x;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) {
    const int r = xrow_c[i];
    roff[i] = r >= 0 ? r * LS : -1;
    tx[i] = twx[i];
  }
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) acc[i] = (TACC)0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int b0 = grp_b * gsize, b1 = min(nbands, b0 + gsize);
  for (int b = b0; b < b1; ++b) {
    const cplx<T>* Sz = S + ((size_t)b * N3 + z) * ncol;
    {
      constexpr int Q = SY::Q, P = SY::P, G = 32 / P;
      const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
      const LaneTw<T, Q, P> lty(ty, p);
      for (int r0 = warp * G; r0 < nxr; r0 += nw * G) {
        const int r = r0 + grp;
        const bool ok = r < nxr;
        const int* so = stick_of + (size_t)(ok ? r : 0) * N2;
        cplx<T> v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int cs = ok ? so[P * q + p] : -1;
          v[q] = cs >= 0 ? Sz[cs] : mk<T>(0, 0);
        }
        if constexpr (LY::kTile) line_inv_tr<T, Q, P>(v, p, lty, tiles + warp * kWT + grp * P * (P + 1), 1, true);
        else line_inv<T, Q, P>(v, p, ty);
        if (ok) {
          cplx<T>* row = Pl + r * LS;
#pragma unroll
          for (int k = 0; k < Q; ++k) row[LY::kTile ? dt_index<Q, P>(p, pr, k) : k + Q * pr] = v[k];
        }
      }
    }
    __syncthreads();
    {
      constexpr int Q = SX::Q, P = SX::P, G = 32 / P;
      const int grp = lane / P, p = lane % P, pr = bitrev_lane<P>(p);
      const LaneTw<T, Q, P> ltx(tx, p);
      const TACC wb = wsq ? (TACC)(wsq[b] * wsq[b]) : (TACC)1;  // the band's occupation weight
      for (int c0 = warp * G; c0 < N2; c0 += nw * G) {
        const int y = c0 + grp;
        const bool ok = y < N2;
        cplx<T> v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int o = roff[P * q + p];
          v[q] = ok && o >= 0 ? Pl[o + y] : mk<T>(0, 0);
        }
        if constexpr (LX::kTile) line_inv_tr<T, Q, P>(v, p, ltx, tiles + warp * kWT + grp * P * (P + 1), 1, true);
        else line_inv<T, Q, P>(v, p, tx);
        if (ok)
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            const TACC re = v[k].x, im = v[k].y;
            acc[(LX::kTile ? dt_index<Q, P>(p, pr, k) : k + Q * pr) * N2 + y] += wb * (re * re + im * im);
          }
      }
    }
    __syncthreads();
  }
  if constexpr (sizeof(TACC) == 4) {  // FP32 sums stored as they are (half the traffic); the caller scales
    float* out = reinterpret_cast<float*>(part) + ((size_t)grp_b * N3 + z) * N1 * N2;
    for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) out[i] = acc[i];
  } else {
    double* out = part + ((size_t)grp_b * N3 + z) * N1 * N2;
    for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) out[i] = (double)acc[i] * wfac;
  }
}

template <typename T, int N, typename TACC>
static size_t density_reg_smem(int nxr) {
  constexpr int kWT = PlaneLines<T, N>::kWarpTile;
  return (size_t)N * N * sizeof(TACC) +
         sizeof(cplx<T>) * (2 * N + PlaneWarps<N>::value * kWT + (size_t)nxr * PlaneStride<N>::value) + N * sizeof(int);
}

template <typename T, int N, typename TACC>
static int density_planes_reg_acc(Ctx* c, const Basis& B, const cplx<T>* S, int nbands, int ngrp, int gsize,
                                  double wfac, const double* wsq, double* part) {
  static int done[64];
  int st;
  if ((st = set_smem_once(c, k_plane_density_reg<T, N, N, TACC>, done))) return st;
  const size_t smem = density_reg_smem<T, N, TACC>(B.nxr);
  k_plane_density_reg<T, N, N, TACC><<<dim3(N, ngrp), 32 * PlaneWarps<N>::value, smem, c->stream>>>(
      S, B.ncol, nbands, gsize, B.d_stick_of, B.d_xrow_c, B.nxr, tw_of<T>(c, 0), tw_of<T>(c, 1), wfac, wsq, part);
  PARO_LAUNCH(c, "k_plane_density_reg");
  return PARO_OK;
}

template <typename T, int N>
static int density_planes_reg_n(Ctx* c, const Basis& B, const cplx<T>* S, int nbands, int ngrp, int gsize,
                                double wfac, const double* wsq, double* part) {
  // FP32 orbitals: the group's |psi|^2 sum in FP32 (an 8-term sum, rounding of the FP32 FFT's own size) keeps
  // the per-point accumulation off GB300's slow FP64 pipe; the groups are summed in FP64 by the caller
  if constexpr (sizeof(T) == 4)
    return density_planes_reg_acc<T, N, float>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
  if (density_reg_smem<T, N, double>(B.nxr) <= 227 * 1024)
    return density_planes_reg_acc<T, N, double>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
  return fail(c, PARO_ERR_ARG, "density: plane too large for shared memory");
}

template <typename T>
int density_planes_reg(Ctx* c, int ik, const cplx<T>* S, int nbands, int ngrp, int gsize, double wfac,
                       const double* wsq, double* part, bool* used, bool* f32part) {
  *used = false;
  *f32part = sizeof(T) == 4;  // FP32 orbitals: unscaled FP32 partial planes (density_planes_reg_n)
  const int n = c->N[0];
  if (c->N[1] != n || c->N[2] != n) return PARO_OK;
  const size_t acc_bytes = (sizeof(T) == 4 && gsize <= 8) ? sizeof(float) : sizeof(double);
  if ((size_t)sizeof(cplx<T>) * (2 * n + n * (n + (n == 72 ? 2 : 1))) + (size_t)n * n * acc_bytes > 227 * 1024)
    return PARO_OK;  // the plane at its PlaneStride and the accumulator
  const Basis& B = c->bases[ik];
  *used = true;
  switch (n) {
    case 32: return density_planes_reg_n<T, 32>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
    case 36: return density_planes_reg_n<T, 36>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
    case 48: return density_planes_reg_n<T, 48>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
    case 72: return density_planes_reg_n<T, 72>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
    case 128: return density_planes_reg_n<T, 128>(c, B, S, nbands, ngrp, gsize, wfac, wsq, part);
    default: *used = false; return PARO_OK;
  }
}

// pass 1 alone (z-inverse of the sticks) with the register FFT; false in *used for other grids
template <typename T>
static int sticks_inverse_reg(Ctx* c, int ik, int nb, const cplx<T>* psi, cplx<T>* S, bool* used) {
  *used = false;
  const int n = c->N[2];
  if (c->N[0] != n || c->N[1] != n) return PARO_OK;
  const Basis& B = c->bases[ik];
  const dim3 gz((B.ncol + kStickBatch - 1) / kStickBatch, nb);
  const size_t smz = (size_t)sizeof(cplx<T>) * (n + kStickBatch * (n + 1));
  static int done[5][64];
  int st = PARO_OK;
  *used = true;
  switch (n) {
#define PARO_ZINV_CASE(NN, I)                                                                                    \
  case NN:                                                                                                      \
    if ((st = set_smem_once(c, k_zpass_inv_reg<T, NN>, done[I]))) return st;                                    \
    k_zpass_inv_reg<T, NN><<<gz, 256, smz, c->stream>>>(psi, B.npw, S, B.d_col_off, B.d_g_col, B.d_g_z, B.ncol, \
                                                        tw_of<T>(c, 2), nullptr, kStickBatch);                  \
    PARO_LAUNCH(c, "k_zpass_inv_reg");                                                                          \
    return PARO_OK;
    PARO_ZINV_CASE(32, 0)
    PARO_ZINV_CASE(36, 1)
    PARO_ZINV_CASE(48, 2)
    PARO_ZINV_CASE(72, 3)
    PARO_ZINV_CASE(128, 4)
#undef PARO_ZINV_CASE
    default:
      *used = false;
      return st;
  }
}
