// 3D lattice (D3Q7): scalar advection, Euler and reactive Euler.
//
// The method of Section 2 in three dimensions (the DdQ(2d+1) lattice of
// Section 2.3 with d = 3; the paper names 3D detonations as future work):
// velocities e_0 = 0, e_j = unit vector j, e_{j+3} = -e_j; speed bounds,
// alpha_j and the step control of Eqs. 2.19/2.21 over three directions; the
// indicator (2.13)/(2.14) summed over three directions and smoothed over the
// 3^3 box (2.15); collision, pull streaming and the implicit moment as in 2D.
//
// Implementation: four kernels over a ghost-extended copy of U (3 ghost
// layers per side, periodic or outflow), the 3D counterpart of the unfused
// 2D path: K0 moments (or, when the previous step's K3 already wrote the
// interior of U, only the ghost layers), K1 indicator, K2 omega, K3
// collision + streaming + implicit moment + side outputs.  Distributions use the row layout of the
// 2D path with rows = z * ny + y, so the row-wise kernels (moments,
// checkpoints) serve 3D lattices unchanged.
#pragma once
#include "common.cuh"
#include "physics.cuh"
#include "fused.cuh"
#include "unfused.cuh"

namespace lbmh {

// primitive variables of a 3D Euler-type state
template <class R>
struct Prim3 {
  R rho, u, v, w, p, c, Y;
};

template <int SYS>
struct Fields3 {
  static constexpr int M = SYS == SYS_ADV ? 1 : (SYS == SYS_EULER ? 5 : 6);
  static constexpr int Q = 7;
};

template <int SYS, class R>
__device__ __forceinline__ Prim3<R> prim3(const Phys<R>& K, const R* U) {
  Prim3<R> w;
  w.rho = w.u = w.v = w.w = w.p = w.c = w.Y = R(0);
  if constexpr (SYS != SYS_ADV) {
    w.rho = U[0];
    const R inv = frcp(w.rho);
    w.u = U[1] * inv;
    w.v = U[2] * inv;
    w.w = U[3] * inv;
    const R kin = R(0.5) * w.rho * (w.u * w.u + w.v * w.v + w.w * w.w);
    R chem = R(0);
    if constexpr (SYS == SYS_REACT) {
      w.Y = U[5] * inv;
      chem = K.q * U[5];
    }
    w.p = K.gm1 * (U[4] - kin - chem);
    w.c = fsqrt(K.gamma * w.p * inv);
  }
  return w;
}

template <class R>
__device__ __forceinline__ R adv3(const Phys<R>& K, const DevParams& P, int dir) {
  if (dir == 0) return K.adv0;
  if (dir == 1) return K.adv1;
  if constexpr (sizeof(R) == 4)
    return P.pf.adv2;
  else
    return P.adv_z;
}

template <int SYS, class R>
__device__ __forceinline__ void flux3(const Phys<R>& K, const DevParams& P, const R* U, const Prim3<R>& w, int dir,
                                      R* F) {
  if constexpr (SYS == SYS_ADV) {
    F[0] = adv3<R>(K, P, dir) * U[0];
  } else {
    // selected, not indexed: dir may be a run-time value (the fused kernel's
    // halo posts), and an indexed array would live in local memory
    const R vn = dir == 0 ? w.u : (dir == 1 ? w.v : w.w);
    F[0] = w.rho * vn;
#pragma unroll
    for (int t = 0; t < 3; t++) F[1 + t] = U[1 + t] * vn + (dir == t ? w.p : R(0));
    F[4] = vn * (U[4] + w.p);
    if constexpr (SYS == SYS_REACT) F[5] = U[5] * vn;
  }
}

template <int SYS, class R>
__device__ __forceinline__ R speed3(const Phys<R>& K, const DevParams& P, const Prim3<R>& w, int dir) {
  if constexpr (SYS == SYS_ADV) {
    return rabs(adv3<R>(K, P, dir));
  } else {
    return rabs(dir == 0 ? w.u : (dir == 1 ? w.v : w.w)) + w.c;
  }
}

// Sum over the characteristic fields of theta^{(r,j)} (Eq. 2.13) along dir:
// closed-form L_j for the Toro-normalised right eigenvectors (acoustic
// (1, u -+ c e_j, H -+ u_j c[, Y]), entropy (1, u, |u|^2/2 [+ qY][, Y]), two
// shear waves (unit tangential velocity), species (0, 0, q, 1)).
template <int SYS, class R>
__device__ __forceinline__ R theta3(const Phys<R>& K, const Prim3<R>& w, int dir, const R* dm, const R* dp) {
  constexpr int M = Fields3<SYS>::M;
  R wm[M], wp[M];
  if constexpr (SYS == SYS_ADV) {
    wm[0] = dm[0];
    wp[0] = dp[0];
  } else {
    const R c = w.c;
    const R inv_c2 = frcp(c * c);
    const R vel[3] = {w.u, w.v, w.w};
    const R q2 = R(0.5) * (w.u * w.u + w.v * w.v + w.w * w.w);
    const R un = vel[dir];
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const R* dU = s == 0 ? dm : dp;
      R* out = s == 0 ? wm : wp;
      R chem = R(0);
      if constexpr (SYS == SYS_REACT) chem = K.q * dU[5];
      const R dpres = K.gm1 * (dU[4] - w.u * dU[1] - w.v * dU[2] - w.w * dU[3] + q2 * dU[0] - chem);
      const R rdun = dU[1 + dir] - un * dU[0];  // rho d(u_n)
      out[0] = R(0.5) * (dpres - c * rdun) * inv_c2;
      out[1] = dU[0] - dpres * inv_c2;
      int r = 2;
#pragma unroll
      for (int t = 0; t < 3; t++)
        if (t != dir) out[r++] = dU[1 + t] - vel[t] * dU[0];  // rho d(u_t)
      if constexpr (SYS == SYS_REACT) out[r++] = dU[5] - w.Y * dU[0];  // rho dY
      out[M - 1] = R(0.5) * (dpres + c * rdun) * inv_c2;
    }
  }
  R nu = R(0);
#pragma unroll
  for (int r = 0; r < M; r++) {
    const R am = rabs(wm[r]), ap = rabs(wp[r]);
    nu += fdiv(rabs(wp[r] - wm[r]), am + ap + K.dx) + am + ap;
  }
  return nu;
}

struct StepCoef3 {
  double dt, lam, alpha[3], a0, aj[3];
  int active;
};

__device__ __forceinline__ StepCoef3 step_coef3(const DevParams& P, const Ctl* ctl, int slot) {
  StepCoef3 c;
  const double ab[3] = {bits_to_double(ctl->amax[slot][0]), bits_to_double(ctl->amax[slot][1]),
                        bits_to_double(ctl->amax_z[slot])};
  const double t = ctl->t[slot];
  c.active = !(P.T > 0.0 && t >= P.T) && !(P.max_steps > 0 && ctl->nsteps[slot] >= P.max_steps);
  c.dt = P.cfl * P.dx / (ab[0] + ab[1] + ab[2]);
  c.lam = P.dx / c.dt;
  double alsum = 0.0;
#pragma unroll
  for (int j = 0; j < 3; j++) {
    c.alpha[j] = ab[j] + P.eps;
    alsum += c.alpha[j];
  }
  c.a0 = 1.0 - alsum / c.lam;
#pragma unroll
  for (int j = 0; j < 3; j++) c.aj[j] = c.alpha[j] / (2.0 * c.lam);
  return c;
}

__device__ __forceinline__ void advance_ctl3(Ctl* ctl, int slot, const StepCoef3& c) {
  const int s1 = (slot + 1) % 3, s2 = (slot + 2) % 3;
  if (c.active) {
    ctl->t[s1] = ctl->t[slot] + c.dt;
    ctl->nsteps[s1] = ctl->nsteps[slot] + 1;
    ctl->parity[s1] = ctl->parity[slot] ^ 1;
    ctl->last_dt = c.dt;
    ctl->last_lambda = c.lam;
  } else {
    ctl->t[s1] = ctl->t[slot];
    ctl->nsteps[s1] = ctl->nsteps[slot];
    ctl->parity[s1] = ctl->parity[slot];
    ctl->amax[s1][0] = ctl->amax[slot][0];
    ctl->amax[s1][1] = ctl->amax[slot][1];
    ctl->amax_z[s1] = ctl->amax_z[slot];
  }
  ctl->amax[s2][0] = ctl->amax[s2][1] = 0ull;
  ctl->amax_z[s2] = 0ull;
}

// ghost-extended 3D geometry: ex x ey x ez nodes, 3 ghost layers per side
// The ghost-extended grid: ex x ey x ez nodes (the lattice plus GH layers on
// every side), stored with rows of px >= ex elements (px a multiple of 4, so
// that every row starts on 16 bytes, as a TMA box needs).  Columns [ex, px)
// are never read or written.
struct ExtGeom3 {
  int ex, ey, ez, px;
  __device__ __forceinline__ long long idx(int ek, int ej, int ei) const {
    return ((long long)ek * ey + ej) * px + ei;
  }
  // elements of one copy of one field
  __host__ __device__ __forceinline__ long long size() const { return (long long)px * ey * ez; }
};
inline int ext_pitch3(int ex) { return (ex + 3) / 4 * 4; }

// offset of node (i, j, k) in a distribution plane (row = k * ny + j)
__device__ __forceinline__ long long cell3(const DevParams& P, int i, int j, int k) {
  return ((long long)k * P.ny3 + j) * P.pitch + i + XPAD;
}

__device__ __forceinline__ double nanmax3(double a, double b) { return (a > b || a != a) ? a : b; }

// block maxima of three speeds into d0..d2 (one atomic per block and value)
__device__ __forceinline__ void block_max3_to(double s0, double s1, double s2, unsigned long long* d0,
                                              unsigned long long* d1, unsigned long long* d2) {
  __shared__ double red[3][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 = nanmax3(s0, __shfl_xor_sync(0xffffffffu, s0, o));
    s1 = nanmax3(s1, __shfl_xor_sync(0xffffffffu, s1, o));
    s2 = nanmax3(s2, __shfl_xor_sync(0xffffffffu, s2, o));
  }
  __syncthreads();
  if (lane == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
    red[2][w] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int i = 0; i < nw; i++) {
      m0 = nanmax3(m0, red[0][i]);
      m1 = nanmax3(m1, red[1][i]);
      m2 = nanmax3(m2, red[2][i]);
    }
    atomic_max_nonneg(d0, m0);
    atomic_max_nonneg(d1, m1);
    atomic_max_nonneg(d2, m2);
  }
}

// speed bound of the FP64 initial state -> ainit (Eq. 2.19)
template <int SYS>
__global__ void __launch_bounds__(kBlock) k3_init_speed(DevParams P, const double* U0, Ctl* ctl) {
  constexpr int M = Fields3<SYS>::M;
  const long long nn = (long long)P.nx * P.ny;
  const Phys<double> K = make_phys<double>(P);
  double s[3] = {0.0, 0.0, 0.0};
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
       node += (long long)gridDim.x * blockDim.x) {
    double U[M];
#pragma unroll
    for (int c = 0; c < M; c++) U[c] = U0[c * nn + node];
    const Prim3<double> w = prim3<SYS, double>(K, U);
#pragma unroll
    for (int d = 0; d < 3; d++) s[d] = nanmax3(s[d], speed3<SYS, double>(K, P, w, d));
  }
  block_max3_to(s[0], s[1], s[2], (unsigned long long*)&ctl->ainit[0], (unsigned long long*)&ctl->ainit[1],
                (unsigned long long*)&ctl->ainit_z);
}

// f := f^eq(U0) with alpha^0, lambda^0 (Eq. 2.20); speed bound of the stored
// state into slot 0
template <int SYS, class R>
__global__ void __launch_bounds__(kBlock) k3_init_eq(DevParams P, const double* U0, R* f, Ctl* ctl) {
  constexpr int M = Fields3<SYS>::M;
  const long long nn = (long long)P.nx * P.ny;
  const double ab[3] = {ctl->ainit[0], ctl->ainit[1], ctl->ainit_z};
  const double dt = P.cfl * P.dx / (ab[0] + ab[1] + ab[2]);
  const double lam = P.dx / dt;
  const double al[3] = {ab[0] + P.eps, ab[1] + P.eps, ab[2] + P.eps};
  const R inv2l = R(1.0 / (2.0 * lam));
  const R alr[3] = {R(al[0]), R(al[1]), R(al[2])};
  const RestCoef<R> rc = rest_coef<R>(1.0 - (al[0] + al[1] + al[2]) / lam, alr, 3, inv2l);
  const Phys<R> K = make_phys<R>(P);
  const long long nf = 7ll * M * P.plane;  // elements of the distributions (index guards)
  double s[3] = {0.0, 0.0, 0.0};
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
       node += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(node / P.nx), i = (int)(node % P.nx);
    const long long off = (long long)row * P.pitch + i + XPAD;
    R U[M];
#pragma unroll
    for (int c = 0; c < M; c++) U[c] = R(U0[c * nn + node]);
    const Prim3<R> w = prim3<SYS, R>(K, U);
#pragma unroll
    for (int c = 0; c < M; c++) f[chk((long long)c * P.plane + off, nf, &ctl->status)] = rest_eq(rc.hi, rc.lo, U[c]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      R F[M];
      flux3<SYS, R>(K, P, U, w, d, F);
#pragma unroll
      for (int c = 0; c < M; c++) {
        f[chk((long long)((1 + d) * M + c) * P.plane + off, nf, &ctl->status)] = (R(al[d]) * U[c] + F[c]) * inv2l;
        f[chk((long long)((4 + d) * M + c) * P.plane + off, nf, &ctl->status)] = (R(al[d]) * U[c] - F[c]) * inv2l;
      }
    }
    // moments of the stored distributions, summed k = 0..6 as a step does
    R Us[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      R sum = R(0);
#pragma unroll
      for (int k = 0; k < 7; k++) sum += f[chk((long long)(k * M + c) * P.plane + off, nf, &ctl->status)];
      Us[c] = sum;
    }
    const Prim3<R> ws = prim3<SYS, R>(K, Us);
#pragma unroll
    for (int d = 0; d < 3; d++) s[d] = nanmax3(s[d], (double)speed3<SYS, R>(K, P, ws, d));
  }
  block_max3_to(s[0], s[1], s[2], &ctl->amax[0][0], &ctl->amax[0][1], &ctl->amax_z[0]);
}

// speed bound of the stored distributions -> slot 0 (after a checkpoint load)
template <int SYS, class R>
__global__ void __launch_bounds__(kBlock) k3_speed_of_f(DevParams P, R* const* buf, Ctl* ctl) {
  constexpr int M = Fields3<SYS>::M;
  const long long nn = (long long)P.nx * P.ny;
  const Phys<R> K = make_phys<R>(P);
  const R* f = buf[ctl->parity[0]];
  double s[3] = {0.0, 0.0, 0.0};
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
       node += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(node / P.nx), i = (int)(node % P.nx);
    const long long off = (long long)row * P.pitch + i + XPAD;
    R U[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      R sum = R(0);
#pragma unroll
      for (int k = 0; k < 7; k++) sum += f[chk((long long)(k * M + c) * P.plane + off, 7ll * M * P.plane, &ctl->status)];
      U[c] = sum;
    }
    const Prim3<R> w = prim3<SYS, R>(K, U);
#pragma unroll
    for (int d = 0; d < 3; d++) s[d] = nanmax3(s[d], (double)speed3<SYS, R>(K, P, w, d));
  }
  block_max3_to(s[0], s[1], s[2], &ctl->amax[0][0], &ctl->amax[0][1], &ctl->amax_z[0]);
}

// the extended-grid kernels run on a grid (ceil(ex / blockDim.x), ey, ez):
// coordinates come from the block indices, without 64-bit divisions
__device__ __forceinline__ bool ext_coords(const ExtGeom3& G, int& ei, int& ej, int& ek, long long& e) {
  ei = blockIdx.x * blockDim.x + threadIdx.x;
  ej = blockIdx.y;
  ek = blockIdx.z;
  e = G.idx(ek, ej, ei);
  return ei < G.ex;
}

// U on the ghost-extended grid lives in two copies [2][m][ez][ey][ex]: copy
// p holds the moments of f buffer p.  The collision kernel writes the
// interior of the other copy (U^{n+1} = sum_k f_k^{n+1}, summed as below), so
// a step normally only refills the ghost layers (k3_ghost_fill); the full
// pass K0 runs after the distributions were set from outside.
template <int M, class T>
__device__ __forceinline__ T* ue_copy(T* Ue, const ExtGeom3& G, int par) {
  return Ue + (long long)par * M * G.size();
}

// K0: U = sum_k f_k on the ghost-extended grid (wrapped / clamped reads).  It
// also runs for a finished lattice, so that the copy is valid afterwards.
template <int SYS, class R>
__global__ void k3_moments_ext(DevParams P, R* const* buf, const Ctl* ctl, int slot, ExtGeom3 G, R* Ue2) {
  constexpr int M = Fields3<SYS>::M;
  const long long n = G.size();
  int ei, ej, ek;
  long long e;
  if (!ext_coords(G, ei, ej, ek, e)) return;
  const int par = ctl->parity[slot];
  const R* f = buf[par];
  R* Ue = ue_copy<M>(Ue2, G, par);
  unsigned int* const stc = (unsigned int*)&ctl->status;  // index guards (bounds-checked builds)
  const long long off = cell3(P, map_index(ei - GH, P.nx, P.bc[0], P.bc[1]), map_index(ej - GH, P.ny3, P.bc[2], P.bc[3]),
                              map_index(ek - GH, P.nz3, P.bc_z[0], P.bc_z[1]));
#pragma unroll
  for (int c = 0; c < M; c++) {
    R sum = R(0);
#pragma unroll
    for (int q = 0; q < 7; q++) sum += f[chk((long long)(q * M + c) * P.plane + off, 7ll * M * P.plane, stc)];
    Ue[chk((long long)c * n + e, (long long)M * n, stc)] = sum;
  }
}

// The ghost layers of U copy p from the mapped interior nodes (periodic wrap
// or outflow clamp, as K0 reads them).  Thread g enumerates the ghost nodes:
// the 2 GH planes of z ghosts, then per interior plane the 2 GH rows of y
// ghosts, then per interior row the 2 GH x ghosts.
template <int SYS, class R>
__global__ void k3_ghost_fill(DevParams P, const Ctl* ctl, int slot, ExtGeom3 G, R* Ue2) {
  constexpr int M = Fields3<SYS>::M;
  const long long n = G.size();
  const long long na = 2LL * GH * G.ey * G.ex, nb = 2LL * GH * G.ex * P.nz3, nc = 2LL * GH * P.ny3 * P.nz3;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= na + nb + nc) return;
  if (P.T > 0.0 && ctl->t[slot] >= P.T) return;
  int ei, ej, ek;
  if (g < na) {
    const long long sl = g / ((long long)G.ey * G.ex), rem = g % ((long long)G.ey * G.ex);
    ek = sl < GH ? (int)sl : P.nz3 + (int)sl;
    ej = (int)(rem / G.ex);
    ei = (int)(rem % G.ex);
  } else if (g < na + nb) {
    const long long h = g - na, per = 2LL * GH * G.ex;
    ek = GH + (int)(h / per);
    const int row = (int)((h % per) / G.ex);
    ej = row < GH ? row : P.ny3 + row;
    ei = (int)((h % per) % G.ex);
  } else {
    const long long h = g - na - nb;
    const long long kr = h / (2 * GH);
    ek = GH + (int)(kr / P.ny3);
    ej = GH + (int)(kr % P.ny3);
    const int sx = (int)(h % (2 * GH));
    ei = sx < GH ? sx : P.nx + sx;
  }
  const int mi = map_index(ei - GH, P.nx, P.bc[0], P.bc[1]), mj = map_index(ej - GH, P.ny3, P.bc[2], P.bc[3]),
            mk = map_index(ek - GH, P.nz3, P.bc_z[0], P.bc_z[1]);
  R* Ue = ue_copy<M>(Ue2, G, ctl->parity[slot]);
  const long long e = G.idx(ek, ej, ei), src = G.idx(mk + GH, mj + GH, mi + GH);
#pragma unroll
  for (int c = 0; c < M; c++)
    Ue[chk((long long)c * n + e, (long long)M * n, (unsigned int*)&ctl->status)] =
        Ue[chk((long long)c * n + src, (long long)M * n, (unsigned int*)&ctl->status)];
}

// threads per block of the extended-grid kernels; planes a thread of the
// omega kernel marches along z
constexpr int kBlock3 = 128;
constexpr int kZ3 = 16;

// K1: nu = sum_j sum_r theta^{(r,j)} one layer inside the extension
template <int SYS, class R>
__global__ void k3_indicator(DevParams P, const Ctl* ctl, int slot, ExtGeom3 G, const R* Ue2, R* nu) {
  constexpr int M = Fields3<SYS>::M;
  const long long n = G.size();
  int ei, ej, ek;
  long long e;
  if (!ext_coords(G, ei, ej, ek, e)) return;
  if (P.T > 0.0 && ctl->t[slot] >= P.T) return;
  const R* Ue = ue_copy<M>(Ue2, G, ctl->parity[slot]);
  if (ei < 1 || ei >= G.ex - 1 || ej < 1 || ej >= G.ey - 1 || ek < 1 || ek >= G.ez - 1) return;
  const Phys<R> K = make_phys<R>(P);
  const long long stride[3] = {1, G.px, (long long)G.px * G.ey};
  unsigned int* const stc = (unsigned int*)&ctl->status;  // index guards (bounds-checked builds)
  R U0[M], dm[M], dp[M];
#pragma unroll
  for (int c = 0; c < M; c++) U0[c] = Ue[chk((long long)c * n + e, (long long)M * n, stc)];
  const Prim3<R> w = prim3<SYS, R>(K, U0);
  R sum = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
#pragma unroll
    for (int c = 0; c < M; c++) {
      dm[c] = U0[c] - Ue[chk((long long)c * n + e - stride[d], (long long)M * n, stc)];
      dp[c] = Ue[chk((long long)c * n + e + stride[d], (long long)M * n, stc)] - U0[c];
    }
    sum += theta3<SYS, R>(K, w, d, dm, dp);
  }
  nu[chk(e, n, stc)] = sum;
}

// K2: omega = 1 + 1/(1 + nu~), nu~ the sum over the 3^3 box (Eq. 2.15, 2.16).
// Grid (ceil(ex / 128), ey, ceil(ez / kZ3)): a thread marches kZ3 planes of
// its (x, y) column and keeps the 3 x 3 windows of nu of the planes k - 1, k,
// k + 1 in registers, so a node costs 9 loads instead of 27.  The 27 terms
// are added as the fused step adds them: the three planes at each (bj, bi)
// first, (nu_{k-1} + nu_k) + nu_{k+1}, then those sums in the order (bj, bi).
template <class R>
__global__ void k3_omega(DevParams P, const Ctl* ctl, int slot, ExtGeom3 G, const R* nu, R* om) {
  const int ei = blockIdx.x * blockDim.x + threadIdx.x, ej = blockIdx.y;
  if (ei < 2 || ei >= G.ex - 2 || ej < 2 || ej >= G.ey - 2) return;
  if (P.T > 0.0 && ctl->t[slot] >= P.T) return;
  const int k0 = max(2, (int)blockIdx.z * kZ3), k1 = min(G.ez - 2, (int)blockIdx.z * kZ3 + kZ3);
  const long long n = G.size();
  unsigned int* const stc = (unsigned int*)&ctl->status;  // index guards (bounds-checked builds)
  if (P.omega_mode == 1) {
    R wf;
    if constexpr (sizeof(R) == 4)
      wf = P.pf.omega_fixed;
    else
      wf = P.omega_fixed;
    for (int ek = k0; ek < k1; ek++) om[chk(G.idx(ek, ej, ei), n, stc)] = wf;
    return;
  }
  R win[3][9];  // nu of planes ek - 1, ek, ek + 1 around (ei, ej)
  auto load_plane = [&](int ek, R* o) {
    const long long b = G.idx(ek, ej, ei);
#pragma unroll
    for (int bj = -1; bj <= 1; bj++)
#pragma unroll
      for (int bi = -1; bi <= 1; bi++) o[(bj + 1) * 3 + bi + 1] = nu[chk(b + (long long)bj * G.px + bi, n, stc)];
  };
  if (k0 < k1) {
    load_plane(k0 - 1, win[0]);
    load_plane(k0, win[1]);
  }
#pragma unroll 1
  for (int ek = k0; ek < k1; ek++) {
    load_plane(ek + 1, win[2]);
    R s = R(0);
#pragma unroll
    for (int q = 0; q < 9; q++) s += (win[0][q] + win[1][q]) + win[2][q];
    om[chk(G.idx(ek, ej, ei), n, stc)] = R(1) + fdiv(R(1), R(1) + s);
#pragma unroll
    for (int q = 0; q < 9; q++) {
      win[0][q] = win[1][q];
      win[1][q] = win[2][q];
    }
  }
}

// source of the 3D systems: Arrhenius on rho*Y (reactive; FP64 in the FP64
// mode, FP32 in the FP32 mode, as in 1D and 2D), none otherwise
template <int SYS, class R>
__device__ __forceinline__ void source3(const Phys<R>& K, const R* U, R* S) {
  constexpr int M = Fields3<SYS>::M;
#pragma unroll
  for (int c = 0; c < M; c++) S[c] = R(0);
  if constexpr (SYS == SYS_REACT) {
    if (K.react) {
      if constexpr (sizeof(R) == 4) {
        S[5] = -arrhenius_f32(K, U[0], U[1] * U[1] + U[2] * U[2] + U[3] * U[3], U[4], U[5]);
      } else {
        const double momsq = (double)U[1] * U[1] + (double)U[2] * U[2] + (double)U[3] * U[3];
        S[5] = R(-arrhenius(K, (double)U[0], momsq, (double)U[4], (double)U[5]));
      }
    }
  }
}

// The FP32 mode's FP64 fallback of the 3D root, out of line like the 2D one.
static __device__ __noinline__ RootF64 react_root3_f64_fallback(float rho, float m1, float m2, float m3, float E,
                                                                float zbar, double dt, double Kc, double gamma,
                                                                double q, double Ti) {
  const double d1 = (double)m1, d2 = (double)m2, d3 = (double)m3;
  return react_root_f64((double)rho, d1 * d1 + d2 * d2 + d3 * d3, (double)E, (double)zbar, 0.5 * dt * Kc,
                        gamma - 1.0, q, Ti);
}

// Eq. (2.8) for rho*Y in 3D: the root z of g(z) = z - zbar + dt/2 R(z).  FP64
// in the FP64 mode; in the FP32 mode FP32 first and FP64 where the FP32
// iteration does not converge.  Returns status bits; z = zbar where no root
// is sought.
template <class R>
__device__ __forceinline__ unsigned react_implicit3(const Phys<R>& K, const R* Ubar, double dt, R hdt, R* z) {
  if constexpr (sizeof(R) == 4) {
    float zf;
    const int rc = react_root_f32<3>(K, Ubar, hdt, &zf);
    if (rc == 0) {
      *z = zf;
      return 0u;
    }
    if (rc == 2) {
      *z = Ubar[5];
      return ST_NOROOT;
    }
    const RootF64 rt = react_root3_f64_fallback(Ubar[0], Ubar[1], Ubar[2], Ubar[3], Ubar[4], Ubar[5], dt, K.K,
                                                K.gamma_d, K.q_d, K.Ti);
    *z = R(rt.z);
    return rt.st;
  } else {
    const double mx = (double)Ubar[1], my = (double)Ubar[2], mz = (double)Ubar[3];
    const RootF64 rt = react_root_f64((double)Ubar[0], mx * mx + my * my + mz * mz, (double)Ubar[4], (double)Ubar[5],
                                      0.5 * dt * K.K, K.gamma_d - 1.0, K.q_d, K.Ti);
    *z = R(rt.z);
    return rt.st;
  }
}

// rows (y) per block of the 3D collision kernel; threads per block, and the
// x nodes a block writes: each warp owns a 32-lane segment along x whose
// lanes 1..30 are written (lanes 0 and 31 are halo)
constexpr int kRows3 = 32;
constexpr int kLanes3 = 128, kSeg3 = 30, kOut3 = (kLanes3 / 32) * kSeg3;

// Side outputs of one warp of the 3D collision kernel, with no block barrier:
// maxima of the three speed bounds, FP64-quality sums of U (FP32: TwoSum
// pairs reduced across the warp, combined in FP64 by lane 0; FP64: plain
// sums) into the warp's own partial slot, status bits.  Lane 0 applies a
// maximum only when it exceeds the stored one (a stale read just costs an
// extra atomic, since the maxima only grow during the step).
template <int M, class R>
__device__ __forceinline__ void warp_side_outputs3(R sp0, R sp1, R sp2, const Acc<R>* acc, Ctl* ctl, int slot1,
                                                   double* dst, unsigned st) {
  const int lane = threadIdx.x & 31;
  double sum[M];
  if constexpr (sizeof(R) == 4) {
    float hi[M], lo[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      hi[c] = acc[c].hi;
      lo[c] = acc[c].lo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int c = 0; c < M; c++) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi[c], o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo[c], o);
        const float s2 = hi[c] + oh, bp = s2 - hi[c];
        const float err = (hi[c] - (s2 - bp)) + (oh - bp);
        hi[c] = s2;
        lo[c] += ol + err;
      }
    }
#pragma unroll
    for (int c = 0; c < M; c++) sum[c] = (double)hi[c] + (double)lo[c];
  } else {
#pragma unroll
    for (int c = 0; c < M; c++) sum[c] = acc[c].value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int c = 0; c < M; c++) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
    }
  }
  double m[3] = {(double)sp0, (double)sp1, (double)sp2};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int d = 0; d < 3; d++) m[d] = nanmax3(m[d], __shfl_xor_sync(0xffffffffu, m[d], o));
  }
  const unsigned wst = __reduce_or_sync(0xffffffffu, st);
  if (lane == 0) {
    unsigned long long* dstm[3] = {&ctl->amax[slot1][0], &ctl->amax[slot1][1], &ctl->amax_z[slot1]};
#pragma unroll
    for (int d = 0; d < 3; d++)
      if (!(bits_to_double(__ldcg(dstm[d])) >= m[d])) atomic_max_nonneg(dstm[d], m[d]);
#pragma unroll
    for (int c = 0; c < M; c++) dst[c] = sum[c];
    if (wst) atomicOr(&ctl->status, wst);
  }
}

// launch shape of the collision kernel per system and precision: resident
// blocks per SM (4, at most 128 registers a thread, for FP32 advection and
// Euler; 2 for reactive Euler and FP64) and whether operands are loaded one
// row ahead.  FP64 (bound by the FP64 pipe) loads them where they are used:
// prefetched doubles would spill.  At 4 blocks FP32 Euler spills a few bytes
// a thread, and still runs faster than at 3 blocks without spills.
template <int SYS, class R>
struct K3Occupancy {
  static constexpr bool prefetch = sizeof(R) == 4;
  static constexpr int blocks = (sizeof(R) == 8 || SYS == SYS_REACT) ? 2 : 4;
};

// post-collision value of direction q at a node with state U (primitives pw,
// source S), relaxation w and distributions fq[M] of that direction (Eq. 2.2
// with half the source)
template <int SYS, class R>
__device__ __forceinline__ void post_q(const Phys<R>& K, const DevParams& P, const R* U, const Prim3<R>& pw,
                                       const R* S, R w, const R* fq, int q, R a0, R a0lo, R alq, R akq, R inv2l,
                                       R hdt, R* out) {
  constexpr int M = Fields3<SYS>::M;
  R F[M];
#pragma unroll
  for (int c = 0; c < M; c++) F[c] = R(0);
  if (q != 0) flux3<SYS, R>(K, P, U, pw, (q - 1) % 3, F);
#pragma unroll
  for (int c = 0; c < M; c++) {
    const R feq = q == 0 ? rest_eq(a0, a0lo, U[c]) : (q <= 3 ? (alq * U[c] + F[c]) * inv2l : (alq * U[c] - F[c]) * inv2l);
    R v = fq[c] - w * (fq[c] - feq);
    if constexpr (SYS == SYS_REACT) {
      if (src_field<SYS, 3>(c)) v += hdt * akq * S[c];
    }
    out[c] = v;
  }
}

// K3: collision with the first half-source (Eq. 2.2), pull streaming, the
// implicit moment (2.8) and the second half-source; writes f^{n+1} and the
// interior of the next U copy (U^{n+1} = sum_k f_k^{n+1}); side
// outputs (three speed bounds, FP64-quality sums, status; one partial-sum
// slot per warp).
//
// Grid (ceil(nx / 120), ceil(ny / kRows3), nz), 128 threads: warp w of block
// bx is a 32-lane segment along x (lane l at x = 120 bx + 30 w - 1 + l) that
// marches the block's rows in y by itself, with no block barrier.  At row r
// every lane computes its own post-collision values for e_0, +-x, +-y once
// (primitives and source once per node); the +-x values pass to the
// neighbouring lanes by warp shuffles, the +-y values stay in the lane's
// registers for rows r +- 1, and row r - 1 is streamed.  The +-z values come
// from the planes k -+ 1 and are computed on the fly (one direction each).
// In FP32 loads run one row ahead: the own operands of row r + 1 are issued
// as soon as row r's posts are formed, the +-z operands of row r once row
// r - 1 is written, so each row waits on one memory latency, already
// overlapped with the other phase.  The prefetched operands cost registers:
// resident blocks per SM are set per system and precision (K3Occupancy).
template <int SYS, class R, class IX>
__global__ void __launch_bounds__(kLanes3, (K3Occupancy<SYS, R>::blocks))
    k3_collide_stream(DevParams P, R* const* buf, Ctl* ctl, int slot, ExtGeom3 G, R* Ue2, const R* om,
                      double* partials) {
  constexpr int M = Fields3<SYS>::M, Q = 7;
  constexpr bool SRC = SYS == SYS_REACT;
  // step coefficients (FP64) and their conversions, by one thread per block
  __shared__ StepCoef3 s_cf;
  __shared__ R s_k[10];  // a0, 1/(2 lambda), dt/2, alpha_0..2, a_1..3, a0lo
  if (threadIdx.x == 0) {
    const StepCoef3 c = step_coef3(P, ctl, slot);
    s_cf = c;
    s_k[0] = R(c.a0);
    s_k[1] = R(1.0 / (2.0 * c.lam));
    s_k[2] = R(0.5 * c.dt);
#pragma unroll
    for (int j = 0; j < 3; j++) {
      s_k[3 + j] = R(c.alpha[j]);
      s_k[6 + j] = R(c.aj[j]);
    }
    const RestCoef<R> rc = rest_coef<R>(c.a0, &s_k[3], 3, s_k[1]);
    s_k[0] = rc.hi;
    s_k[9] = rc.lo;
  }
  __syncthreads();
  const StepCoef3 cf = s_cf;
  const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (!cf.active) {
    if (bid == 0 && threadIdx.x == 0) advance_ctl3(ctl, slot, cf);
    return;
  }
  const int par = ctl->parity[slot];
  const R* f = buf[par];
  R* fo = buf[par ^ 1];
  const R* Ue = ue_copy<M>(Ue2, G, par);
  R* Uo_ext = ue_copy<M>(Ue2, G, par ^ 1);  // U^{n+1} of the interior, for the next step
  // offsets in IX: int where every offset of the lattice fits (chosen at launch), else long long
  const IX n = (IX)G.size(), pl = (IX)P.plane;
  const long long nf = 7ll * M * P.plane;  // elements of the distributions (index guards)
  unsigned int* const stc = &ctl->status;
  auto eidx = [&](int ek, int ej, int ei) -> IX { return ((IX)ek * G.ey + ej) * G.px + ei; };
  auto fidx = [&](int ci, int cj, int ck) -> IX { return ((IX)ck * P.ny3 + cj) * P.pitch + ci + XPAD; };
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kOut3 + w * kSeg3 - 1 + lane, k = blockIdx.z;
  const bool out_lane = lane >= 1 && lane <= kSeg3 && i < P.nx;
  const bool halo_or_out = i <= P.nx;  // lanes past x = nx are never read (and lie outside the extension)
  const int mi = map_index(i, P.nx, P.bc[0], P.bc[1]);
  const int mkm = map_index(k - 1, P.nz3, P.bc_z[0], P.bc_z[1]), mkp = map_index(k + 1, P.nz3, P.bc_z[0], P.bc_z[1]);
  const Phys<R> K = make_phys<R>(P);
  const R a0 = s_k[0], a0lo = s_k[9], inv2l = s_k[1], hdt = s_k[2];
  const R al[3] = {s_k[3], s_k[4], s_k[5]};
  const R aj[3] = {s_k[6], s_k[7], s_k[8]};
  R sp0 = R(0), sp1 = R(0), sp2 = R(0);
  Acc<R> acc[M];
#pragma unroll
  for (int c = 0; c < M; c++) acc[c].init();
  unsigned st = 0u;
  const int j0 = blockIdx.y * kRows3, j1 = min(j0 + kRows3, P.ny3);
  // own operands of a row (U, omega, f of e_0, +x, -x, +y, -y at the lane's
  // node; ghost rows: the mapped node, A6), loaded one row ahead
  R oU[M], ow, of[5][M];
  auto load_own = [&](int r) {
    const IX e = eidx(k + GH, r + GH, i + GH);
    const IX off = fidx(mi, map_index(r, P.ny3, P.bc[2], P.bc[3]), k);
#pragma unroll
    for (int c = 0; c < M; c++) oU[c] = halo_or_out ? Ue[chk((IX)c * n + e, (long long)M * n, stc)] : R(1);
    ow = halo_or_out ? om[chk(e, n, stc)] : R(1);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const int qq = q == 0 ? 0 : (q == 1 ? 1 : (q == 2 ? 4 : (q == 3 ? 2 : 5)));  // 0, +x, -x, +y, -y
#pragma unroll
      for (int c = 0; c < M; c++) of[q][c] = halo_or_out ? f[chk((IX)(qq * M + c) * pl + off, nf, stc)] : R(0);
    }
  };
  // operands of the +-z posts of an output row: U, omega and f_{+z} at plane
  // k - 1, U, omega and f_{-z} at plane k + 1
  R zU[2][M], zw[2], zf[2][M];
  auto load_z = [&](int y) {
    const int my = map_index(y, P.ny3, P.bc[2], P.bc[3]);
#pragma unroll
    for (int s2 = 0; s2 < 2; s2++) {
      const int kk = s2 == 0 ? k - 1 : k + 1, qq = s2 == 0 ? 3 : 6;
      const IX ez = eidx(kk + GH, y + GH, i + GH);
      const IX offz = fidx(mi, my, s2 == 0 ? mkm : mkp);
#pragma unroll
      for (int c = 0; c < M; c++) {
        zU[s2][c] = Ue[chk((IX)c * n + ez, (long long)M * n, stc)];
        zf[s2][c] = f[chk((IX)(qq * M + c) * pl + offz, nf, stc)];
      }
      zw[s2] = om[chk(ez, n, stc)];
    }
  };
  // lane registers: post_0, post_{+y} and the received F_{+x}, F_{-x} of row
  // r-1, post_{+y} of row r-2
  R p0_prev[M], py_prev[M], py_prev2[M], fxp_prev[M], fxm_prev[M];
#pragma unroll
  for (int c = 0; c < M; c++) p0_prev[c] = py_prev[c] = py_prev2[c] = fxp_prev[c] = fxm_prev[c] = R(0);
  constexpr bool PF = K3Occupancy<SYS, R>::prefetch;
  if constexpr (PF) load_own(j0 - 1);
#pragma unroll 1
  for (int r = j0 - 1; r <= j1; r++) {
    if constexpr (!PF) load_own(r);
    // own post-collision values of row r
    R p0[M], ppx[M], pmx[M], ppy[M], pmy[M];
    {
      const Prim3<R> pw = prim3<SYS, R>(K, oU);
      R S[M];
      if constexpr (SRC) source3<SYS, R>(K, oU, S);
#pragma unroll
      for (int q = 0; q < 5; q++) {
        const int qq = q == 0 ? 0 : (q == 1 ? 1 : (q == 2 ? 4 : (q == 3 ? 2 : 5)));
        const int dir = qq == 0 ? 0 : (qq - 1) % 3;
        R* o = q == 0 ? p0 : (q == 1 ? ppx : (q == 2 ? pmx : (q == 3 ? ppy : pmy)));
        post_q<SYS, R>(K, P, oU, pw, S, ow, of[q], qq, a0, a0lo, al[dir], qq == 0 ? a0 : aj[dir], inv2l, hdt, o);
      }
    }
    if constexpr (PF) {
      if (r < j1) load_own(r + 1);
    }
    // F_{+x}(x) = post_{+x}(x - e_x) from lane - 1, F_{-x}(x) = post_{-x}(x + e_x)
    // from lane + 1 (lanes 0 and 31 receive their own value and write nothing)
    R fxp[M], fxm[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      fxp[c] = __shfl_up_sync(0xffffffffu, ppx[c], 1);
      fxm[c] = __shfl_down_sync(0xffffffffu, pmx[c], 1);
    }
    const int y = r - 1;
    if (y >= j0 && y < j1 && out_lane) {
      R Fk[Q][M];
#pragma unroll
      for (int c = 0; c < M; c++) {
        Fk[0][c] = p0_prev[c];
        Fk[1][c] = fxp_prev[c];
        Fk[4][c] = fxm_prev[c];
        Fk[2][c] = py_prev2[c];  // post_{+y} of row y - 1
        Fk[5][c] = pmy[c];       // post_{-y} of row y + 1
      }
      // +-z: post_{+z} at plane k - 1, post_{-z} at plane k + 1 (operands
      // loaded in the previous iteration, or here without prefetch)
      if constexpr (!PF) load_z(y);
#pragma unroll
      for (int s2 = 0; s2 < 2; s2++) {
        const int qq = s2 == 0 ? 3 : 6;
        const Prim3<R> pz = prim3<SYS, R>(K, zU[s2]);
        R Sz[M];
        if constexpr (SRC) source3<SYS, R>(K, zU[s2], Sz);
        post_q<SYS, R>(K, P, zU[s2], pz, Sz, zw[s2], zf[s2], qq, a0, a0lo, al[2], aj[2], inv2l, hdt, Fk[qq]);
      }
      R Ubar[M];
#pragma unroll
      for (int c = 0; c < M; c++) {
        R sum = R(0);
#pragma unroll
        for (int q = 0; q < Q; q++) sum += Fk[q][c];
        Ubar[c] = sum;
      }
      // the second half-source dt/2 a_q S(U^{n+1}): Eq. (2.8) makes
      // dt/2 S_5(U^{n+1}) = (rho Y)^{n+1} - (rho Y)bar, so S is not evaluated again
      R hs = R(0);
      if constexpr (SRC) {
        if (K.react && Ubar[5] != R(0)) {
          R z;
          st |= react_implicit3<R>(K, Ubar, cf.dt, hdt, &z);
          hs = z - Ubar[5];
        }
      }
      const IX oo = fidx(i, y, k);
      R Uo[M];
#pragma unroll
      for (int c = 0; c < M; c++) Uo[c] = R(0);
#pragma unroll
      for (int q = 0; q < Q; q++) {
        const R akq = q == 0 ? a0 : aj[(q - 1) % 3];
#pragma unroll
        for (int c = 0; c < M; c++) {
          R v = Fk[q][c];
          if constexpr (SRC) {
            if (src_field<SYS, 3>(c)) v += akq * hs;
          }
          fo[chk((IX)(q * M + c) * pl + oo, nf, stc)] = v;
          Uo[c] += v;
        }
      }
      const IX eo = eidx(k + GH, y + GH, i + GH);
#pragma unroll
      for (int c = 0; c < M; c++) Uo_ext[chk((IX)c * n + eo, (long long)M * n, stc)] = Uo[c];
      const Prim3<R> wn = prim3<SYS, R>(K, Uo);
      sp0 = rmax(sp0, speed3<SYS, R>(K, P, wn, 0));
      sp1 = rmax(sp1, speed3<SYS, R>(K, P, wn, 1));
      sp2 = rmax(sp2, speed3<SYS, R>(K, P, wn, 2));
#pragma unroll
      for (int c = 0; c < M; c++) acc[c].add(Uo[c]);
      bool bad = false;
#pragma unroll
      for (int c = 0; c < M; c++) bad |= !(Uo[c] == Uo[c]);
      if constexpr (SYS != SYS_ADV) bad |= !(wn.rho > R(0)) || !(wn.p > R(0));
      if (bad) st |= ST_NONPHYSICAL;
    }
    // the +-z operands of row r, used when row r is streamed (next iteration)
    if constexpr (PF) {
      if (r >= j0 && r < j1 && out_lane) load_z(r);
    }
#pragma unroll
    for (int c = 0; c < M; c++) {
      py_prev2[c] = py_prev[c];
      py_prev[c] = ppy[c];
      p0_prev[c] = p0[c];
      fxp_prev[c] = fxp[c];
      fxm_prev[c] = fxm[c];
    }
  }
  // side outputs per warp (partial slot bid * 4 + w): no block barrier, so a
  // warp that finished its rows does not wait for the others
  warp_side_outputs3<M, R>(sp0, sp1, sp2, acc, ctl, (slot + 1) % 3, partials + (bid * (kLanes3 / 32) + w) * M, st);
  if (bid == 0 && threadIdx.x == 0) advance_ctl3(ctl, slot, cf);
}

// whether every offset the collision kernel forms fits in an int: Q m planes
// of f and m copies of the extended U (two U copies are addressed from the
// copy's own base)
inline bool k3_offsets_fit_int(const DevParams& P, int m, long long next) {
  const long long lim = 2147483647LL;
  return 7LL * m * P.plane < lim && (long long)m * next < lim;
}

// launch shapes of the 3D kernels
inline dim3 grid3_ext(int ex, int ey, int ez) { return dim3((unsigned)((ex + kBlock3 - 1) / kBlock3), ey, ez); }
inline dim3 grid3_omega(int ex, int ey, int ez) {
  return dim3((unsigned)((ex + kBlock3 - 1) / kBlock3), ey, (unsigned)((ez + kZ3 - 1) / kZ3));
}
inline dim3 grid3_nodes(int nx, int ny, int nz) {
  return dim3((unsigned)((nx + kOut3 - 1) / kOut3), (unsigned)((ny + kRows3 - 1) / kRows3), nz);
}

}  // namespace lbmh
