// Unfused reference step: four simple kernels per time step, one thread per
// node, every intermediate in global scratch.  It is the plain per-grid path
// the fused kernel is measured against, and a second GPU implementation for
// debugging.  Scratch (ghost-extended, 3 layers): U_ext[m][ey][ex],
// nu_ext[ey][ex], om_ext[ey][ex].
#pragma once
#include "physics.cuh"

namespace lbmh {

constexpr int GH = 3;  // ghost layers: the update of one node reads f^n up to 3 nodes away

struct ExtGeom {
  int ex, ey, gy;  // extended sizes; gy = ghost rows (0 in 1D)
  int ez = 1;      // 3D only: extended size in z
  __device__ __forceinline__ long long idx(int ej, int ei) const { return (long long)ej * ex + ei; }
};

template <class R>
__device__ __forceinline__ const R* state_in(R* const* buf, const Ctl* ctl, int slot) {
  return buf[ctl->parity[slot]];
}

// K0: U = sum_k f_k (Eq. 2.3) on every node of the ghost-extended grid, f read
// at the wrapped / clamped index.
template <int SYS, int D, class R>
__global__ void k_moments_ext(DevParams P, R* const* buf, const Ctl* ctl, int slot, ExtGeom G, R* Ue) {
  unsigned int* const stc = (unsigned int*)&ctl->status;  // index guards (bounds-checked builds)
  constexpr int M = Fields<SYS, D>::M, Q = Fields<SYS, D>::Q;
  long long n = (long long)G.ex * G.ey;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (P.T > 0.0 && ctl->t[slot] >= P.T) return;
  const R* f = state_in(buf, ctl, slot);
  int ej = (int)(e / G.ex), ei = (int)(e % G.ex);
  int i = map_index(ei - GH, P.nx, P.bc[0], P.bc[1]);
  int j = D == 2 ? map_index(ej - G.gy, P.ny, P.bc[2], P.bc[3]) : 0;
  long long off = cell(P, i, j);
  R U[M];
#pragma unroll
  for (int c = 0; c < M; c++) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < Q; k++) s += f[chk((long long)(k * M + c) * P.plane + off, (long long)Q * M * P.plane, stc)];
    U[c] = s;
  }
  if (P.has_special_bc) {
    // the moments of the ghost distributions of the fused kernels: a
    // reflecting ghost has the mirror state with the normal momentum
    // reversed, an inflow ghost the inflow state
    const int xs = ghost_side(ei - GH, P.nx, P.bc[0], P.bc[1]);
    const int ys = D == 2 ? ghost_side(ej - G.gy, P.ny, P.bc[2], P.bc[3]) : -1;
    constexpr bool momentum = SYS == SYS_EULER || SYS == SYS_SWE || SYS == SYS_REACT;
    if (xs == BC_INFLOW || ys == BC_INFLOW) {
#pragma unroll
      for (int c = 0; c < M; c++) U[c] = sizeof(R) == 4 ? R(P.pf.u_in[c]) : R(P.u_in[c]);
    } else if constexpr (momentum) {
      if (xs == BC_REFLECT) U[1] = -U[1];
      if (D == 2 && ys == BC_REFLECT) U[2] = -U[2];
    }
  }
#pragma unroll
  for (int c = 0; c < M; c++) Ue[chk((long long)c * n + e, (long long)M * n, stc)] = U[c];
}

// K1: nu = sum_j sum_r theta^{(r,j)} (Eq. 2.10/2.14) one layer inside the extension
template <int SYS, int D, class R>
__global__ void k_indicator(DevParams P, const Ctl* ctl, int slot, ExtGeom G, const R* Ue, R* nu) {
  unsigned int* const stc = (unsigned int*)&ctl->status;  // index guards (bounds-checked builds)
  constexpr int M = Fields<SYS, D>::M;
  long long n = (long long)G.ex * G.ey;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (P.T > 0.0 && ctl->t[slot] >= P.T) return;
  int ej = (int)(e / G.ex), ei = (int)(e % G.ex);
  if (ei < 1 || ei >= G.ex - 1) return;
  if (D == 2 && (ej < 1 || ej >= G.ey - 1)) return;
  const Phys<R> K = make_phys<R>(P);
  R U0[M], dm[M], dp[M];
#pragma unroll
  for (int c = 0; c < M; c++) U0[c] = Ue[chk((long long)c * n + e, (long long)M * n, stc)];
  Prim<R> w = primitives<SYS, D, R>(K, U0);
  R s = R(0);
#pragma unroll
  for (int dir = 0; dir < D; dir++) {
    long long step = dir == 0 ? 1 : G.ex;
#pragma unroll
    for (int c = 0; c < M; c++) {
      dm[c] = U0[c] - Ue[chk((long long)c * n + e - step, (long long)M * n, stc)];
      dp[c] = Ue[chk((long long)c * n + e + step, (long long)M * n, stc)] - U0[c];
    }
    s += theta_sum<SYS, D, R>(K, w, dir, dm, dp);
  }
  nu[chk(e, n, stc)] = s;
}

// K2: omega = 1 + 1/(1 + nu~), nu~ the sum over the 3^d box (Eq. 2.11/2.15, 2.12/2.16)
template <int D, class R>
__global__ void k_omega(DevParams P, const Ctl* ctl, int slot, ExtGeom G, const R* nu, R* om) {
  unsigned int* const stc = (unsigned int*)&ctl->status;  // index guards (bounds-checked builds)
  long long n = (long long)G.ex * G.ey;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (P.T > 0.0 && ctl->t[slot] >= P.T) return;
  int ej = (int)(e / G.ex), ei = (int)(e % G.ex);
  if (ei < 2 || ei >= G.ex - 2) return;
  if (D == 2 && (ej < 2 || ej >= G.ey - 2)) return;
  R w;
  if (P.omega_mode == 1) {
    w = R(P.omega_fixed);
  } else {
    R s = R(0);
    for (int bj = (D == 2 ? -1 : 0); bj <= (D == 2 ? 1 : 0); bj++)
      for (int bi = -1; bi <= 1; bi++) s += nu[chk(e + (long long)bj * G.ex + bi, n, stc)];
    w = R(1) + fdiv(R(1), R(1) + s);
  }
  if (P.sponge_width > 0.0) {  // blended toward 1 over the sponge (x-lo)
    const double r = (double)(ei - GH) + 0.5;
    const double x = r * P.sponge_dx_over_w;
    const double keep = x <= 0.0 ? 0.0 : (x >= 1.0 ? 1.0 : 1.0 - 0.5 * (1.0 + cos(3.14159265358979323846 * x)));
    w = R(1) + (w - R(1)) * R(keep);
  }
  om[chk(e, n, stc)] = w;
}

// velocity e_k of the DdQ(2d+1) lattice: e_0 = 0, e_j = unit j, e_{j+d} = -e_j
template <int D>
__device__ __forceinline__ void lattice_vel(int k, int& ex, int& ey) {
  ex = 0;
  ey = 0;
  if (k == 0) return;
  int j = (k - 1) % D;
  int sg = k <= D ? 1 : -1;
  if (j == 0) ex = sg; else ey = sg;
}

// Block-level reduction of the side outputs: max speeds -> control slot,
// FP64 sums of U^{n+1} -> per-block partials (fixed order, reproducible)
template <int M>
__device__ __forceinline__ void block_side_outputs_to(double sp0, double sp1, const double* usum, Ctl* ctl,
                                                      int slot1, double* dst, unsigned st);

template <int M>
__device__ __forceinline__ void block_side_outputs(double sp0, double sp1, const double* usum, Ctl* ctl, int slot1,
                                                   double* partials, unsigned st) {
  block_side_outputs_to<M>(sp0, sp1, usum, ctl, slot1, partials + (long long)blockIdx.x * M, st);
}

// as block_side_outputs, the block's FP64 sums going to dst[0..M)
template <int M>
__device__ __forceinline__ void block_side_outputs_to(double sp0, double sp1, const double* usum, Ctl* ctl,
                                                      int slot1, double* dst, unsigned st) {
  __shared__ double s_red[32][M + 2];
  __shared__ unsigned s_st;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x == 0) s_st = 0u;
  double v[M + 2];
  v[0] = sp0;
  v[1] = sp1;
#pragma unroll
  for (int c = 0; c < M; c++) v[2 + c] = usum[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] = fmax(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
    v[1] = fmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
#pragma unroll
    for (int c = 0; c < M; c++) v[2 + c] += __shfl_xor_sync(0xffffffffu, v[2 + c], o);
  }
  __syncthreads();
  if (st) atomicOr(&s_st, st);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < M + 2; c++) s_red[wid][c] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double m0 = 0.0, m1 = 0.0, acc[M];
#pragma unroll
    for (int c = 0; c < M; c++) acc[c] = 0.0;
    for (int w2 = 0; w2 < nw; w2++) {
      // NaN-propagating max (a NaN speed marks a non-physical state)
      m0 = (s_red[w2][0] > m0 || s_red[w2][0] != s_red[w2][0]) ? s_red[w2][0] : m0;
      m1 = (s_red[w2][1] > m1 || s_red[w2][1] != s_red[w2][1]) ? s_red[w2][1] : m1;
#pragma unroll
      for (int c = 0; c < M; c++) acc[c] += s_red[w2][2 + c];
    }
    atomic_max_nonneg(&ctl->amax[slot1][0], m0);
    atomic_max_nonneg(&ctl->amax[slot1][1], m1);
#pragma unroll
    for (int c = 0; c < M; c++) dst[c] = acc[c];
    if (s_st) atomicOr(&ctl->status, s_st);
  }
}

// K3: collision with the first half-source at x - e_k, pull streaming, the
// implicit moment (2.8) and the second half-source at x; writes f^{n+1}.
template <int SYS, int D, class R>
__global__ void k_collide_stream(DevParams P, R* const* buf, Ctl* ctl, int slot, ExtGeom G, const R* Ue,
                                 const R* om, double* partials) {
  constexpr int M = Fields<SYS, D>::M, Q = Fields<SYS, D>::Q;
  unsigned int* const stc = &ctl->status;  // index guards (bounds-checked builds)
  const StepCoef cf = step_coef<D>(P, ctl, slot);
  if (!cf.active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) advance_ctl<D>(ctl, slot, cf);
    return;
  }
  const R* f = buf[ctl->parity[slot]];
  R* fo = buf[ctl->parity[slot] ^ 1];
  long long nn = (long long)P.nx * P.ny;
  long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long next = (long long)G.ex * G.ey;
  double sp0 = 0.0, sp1 = 0.0, usum[M];
#pragma unroll
  for (int c = 0; c < M; c++) usum[c] = 0.0;
  unsigned st = 0u;
  const Phys<R> K = make_phys<R>(P);
  const R inv2l = R(1.0 / (2.0 * cf.lam)), hdt = R(0.5 * cf.dt);
  const R al[2] = {R(cf.alpha[0]), R(cf.alpha[1])};
  const R ak[3] = {R(cf.a0), R(cf.aj[0]), R(cf.aj[1])};
  const RestCoef<R> rc = rest_coef<R>(cf.a0, al, D, inv2l);
  if (node < nn) {
    int j = (int)(node / P.nx), i = (int)(node % P.nx);
    R Fk[Q][M];
#pragma unroll
    for (int k = 0; k < Q; k++) {
      int ekx, eky;
      lattice_vel<D>(k, ekx, eky);
      int ei = i + GH - ekx, ej = j + G.gy - eky;  // extended coordinates of x - e_k
      long long e = G.idx(ej, ei);
      R U[M], S[M];
#pragma unroll
      for (int c = 0; c < M; c++) U[c] = Ue[chk((long long)c * next + e, (long long)M * next, stc)];
      int si = map_index(ei - GH, P.nx, P.bc[0], P.bc[1]);
      int sj = D == 2 ? map_index(ej - G.gy, P.ny, P.bc[2], P.bc[3]) : 0;
      Prim<R> w = primitives<SYS, D, R>(K, U);
      R feq[M];
      if (k == 0) {
#pragma unroll
        for (int c = 0; c < M; c++) feq[c] = rest_eq(rc.hi, rc.lo, U[c]);
      } else {
        int jd = (k - 1) % D;
        R F[M];
        flux<SYS, D, R>(K, U, w, jd, F);
        R sg = k <= D ? R(1) : R(-1);
#pragma unroll
        for (int c = 0; c < M; c++) feq[c] = (al[jd] * U[c] + sg * F[c]) * inv2l;
      }
      source<SYS, D, R>(K, U, K.xb + R(si) * K.dx, K.yb + R(sj) * K.dx, S);
      R wk = om[chk(e, next, stc)];
      R akk = k == 0 ? ak[0] : ak[1 + (k - 1) % D];
      long long off = cell(P, si, sj);
#pragma unroll
      for (int c = 0; c < M; c++) {
        R fk = f[chk((long long)(k * M + c) * P.plane + off, (long long)Q * M * P.plane, stc)];
        R v = fk - wk * (fk - feq[c]);
        if (src_field<SYS, D>(c)) v += hdt * akk * S[c];
        Fk[k][c] = v;
      }
    }
    R Ubar[M], Un[M], Sn[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < Q; k++) s += Fk[k][c];
      Ubar[c] = s;
    }
    const R xn = K.xb + R(i) * K.dx, yn = K.yb + R(j) * K.dx;
    st |= implicit_moment<SYS, D, R>(K, Ubar, xn, yn, cf.dt, hdt, Un);
    // the second half-source dt/2 a_k S(U^{n+1}): reactive Euler takes it
    // from Eq. (2.8), dt/2 S(U^{n+1}) = U^{n+1} - Ubar, without evaluating S
    // again; the other systems evaluate S(U^{n+1})
    if constexpr (SYS != SYS_REACT) source<SYS, D, R>(K, Un, xn, yn, Sn);
    long long off = cell(P, i, j);
    R Us[M];
#pragma unroll
    for (int c = 0; c < M; c++) Us[c] = R(0);
#pragma unroll
    for (int k = 0; k < Q; k++) {
      R akk = k == 0 ? ak[0] : ak[1 + (k - 1) % D];
#pragma unroll
      for (int c = 0; c < M; c++) {
        R v = Fk[k][c];
        if constexpr (SYS == SYS_REACT) {
          if (src_field<SYS, D>(c)) v += akk * (Un[c] - Ubar[c]);
        } else {
          v += hdt * akk * Sn[c];
        }
        fo[chk((long long)(k * M + c) * P.plane + off, (long long)Q * M * P.plane, stc)] = v;
        Us[c] += v;  // the moments the next step will see (Eq. 2.3, k = 0..Q-1)
      }
    }
    Prim<R> wn = primitives<SYS, D, R>(K, Us);
    sp0 = (double)max_speed<SYS, D, R>(K, wn, 0);
    if (D == 2) sp1 = (double)max_speed<SYS, D, R>(K, wn, 1);
#pragma unroll
    for (int c = 0; c < M; c++) usum[c] = (double)Us[c];
    st |= state_status<SYS, D, R>(Us, wn);
  }
  block_side_outputs<M>(sp0, sp1, usum, ctl, (slot + 1) % 3, partials, st);
  if (blockIdx.x == 0 && threadIdx.x == 0) advance_ctl<D>(ctl, slot, cf);
}

}  // namespace lbmh
