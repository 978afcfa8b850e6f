// Per-node physics of the four systems on the hot path, templated on the
// system, the dimension and the arithmetic type R (float or double):
// flux F_j(U), the speed bound max_r |lambda_r(dF_j/dU)|, the characteristic
// smoothness indicator, the source S(U) and the implicit moment of Eq. (2.8).
#pragma once
#include "common.cuh"

namespace lbmh {

template <class R> __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
__device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float rexp_(float x) { return expf(x); }
__device__ __forceinline__ double rexp_(double x) { return exp(x); }

// Primitive variables of an Euler-type or shallow-water state.
template <class R>
struct Prim {
  R rho, u, v, p, c, Y;  // Euler / reactive; for shallow water rho holds h
  bool dry;
};

template <int SYS, int D, class R>
__device__ __forceinline__ Prim<R> primitives(const DevParams& P, const R* U) {
  Prim<R> w;
  w.Y = R(0);
  w.dry = false;
  if constexpr (SYS == SYS_EULER || SYS == SYS_REACT) {
    w.rho = U[0];
    R inv = R(1) / w.rho;
    w.u = U[1] * inv;
    w.v = D == 2 ? U[2] * inv : R(0);
    R kin = R(0.5) * w.rho * (w.u * w.u + w.v * w.v);
    R chem = R(0);
    if constexpr (SYS == SYS_REACT) {
      w.Y = U[D + 2] * inv;
      chem = R(P.q) * U[D + 2];
    }
    w.p = R(P.gamma - 1.0) * (U[D + 1] - kin - chem);
    w.c = rsqrt_(R(P.gamma) * w.p / w.rho);
  } else if constexpr (SYS == SYS_SWE) {
    w.rho = U[0];
    w.dry = w.rho < R(P.h_dry);
    if (w.dry) {
      w.u = R(0);
      w.v = R(0);
    } else {
      R inv = R(1) / w.rho;
      w.u = U[1] * inv;
      w.v = D == 2 ? U[2] * inv : R(0);
    }
    w.c = rsqrt_(R(P.g) * (w.rho > R(0) ? w.rho : R(0)));
    w.p = R(0);
  } else {
    w.rho = w.u = w.v = w.p = w.c = R(0);
  }
  return w;
}

// Flux F_dir(U): Section 5 (shallow water, reactive Euler; Euler is the
// reactive flux without species).
template <int SYS, int D, class R>
__device__ __forceinline__ void flux(const DevParams& P, const R* U, const Prim<R>& w, int dir, R* F) {
  if constexpr (SYS == SYS_ADV) {
    F[0] = R(P.adv[dir]) * U[0];
  } else if constexpr (SYS == SYS_SWE) {
    R vn = dir == 0 ? w.u : w.v;
    R pres = R(0.5) * R(P.g) * w.rho * w.rho;
    F[0] = w.rho * vn;
    F[1] = w.rho * w.u * vn + (dir == 0 ? pres : R(0));
    if constexpr (D == 2) F[2] = w.rho * w.v * vn + (dir == 1 ? pres : R(0));
  } else {
    R vn = dir == 0 ? w.u : w.v;
    F[0] = w.rho * vn;
    F[1] = w.rho * w.u * vn + (dir == 0 ? w.p : R(0));
    if constexpr (D == 2) F[2] = w.rho * w.v * vn + (dir == 1 ? w.p : R(0));
    F[D + 1] = vn * (U[D + 1] + w.p);
    if constexpr (SYS == SYS_REACT) F[D + 2] = U[D + 2] * vn;
  }
}

// max_r |lambda_r(dF_dir/dU)|, the inner maximum of Eq. (2.17)/(2.19)
template <int SYS, int D, class R>
__device__ __forceinline__ R max_speed(const DevParams& P, const Prim<R>& w, int dir) {
  if constexpr (SYS == SYS_ADV) {
    return rabs(R(P.adv[dir]));
  } else {
    R vn = dir == 0 ? w.u : w.v;
    return rabs(vn) + w.c;
  }
}

// Sum over the m characteristic fields of theta^{(r,j)} (Eq. 2.9/2.13) at a
// node with state U0, backward difference dm = U0 - U_{i-n_j} and forward
// difference dp = U_{i+n_j} - U0.  L_j(U0) is applied in closed form: the
// increments are converted to primitive increments at U0 and decomposed on
// the right eigenvectors (1, u-c, v, H-uc[, Y]), (1, u, v, |u|^2/2[+qY][, Y]),
// (0, 0, 1, v[, 0]), (0, 0, 0, q, 1), (1, u+c, v, H+uc[, Y]) (Euler-type) or
// (1, u-c, v), (0, 0, 1), (1, u+c, v) (shallow water), rotated for dir = y.
template <int SYS, int D, class R>
__device__ __forceinline__ R theta_sum(const DevParams& P, const Prim<R>& w, int dir, const R* dm,
                                       const R* dp, R dx) {
  constexpr int M = Fields<SYS, D>::M;
  R wm[M], wp[M];
  if constexpr (SYS == SYS_ADV) {
    wm[0] = dm[0];
    wp[0] = dp[0];
  } else if constexpr (SYS == SYS_SWE) {
    R c = w.c;
    R cmin = rsqrt_(R(P.g) * R(P.h_dry));
    c = c < cmin ? cmin : c;
    R inv_c = R(1) / c;
    R un = dir == 0 ? w.u : w.v;
    R hdn_m = dm[1 + dir] - un * dm[0];  // h d(u_n)
    R hdn_p = dp[1 + dir] - un * dp[0];
    wm[0] = R(0.5) * (dm[0] - hdn_m * inv_c);
    wp[0] = R(0.5) * (dp[0] - hdn_p * inv_c);
    if constexpr (D == 2) {
      R ut = dir == 0 ? w.v : w.u;
      wm[1] = dm[2 - dir] - ut * dm[0];  // h d(u_t)
      wp[1] = dp[2 - dir] - ut * dp[0];
    }
    wm[M - 1] = R(0.5) * (dm[0] + hdn_m * inv_c);
    wp[M - 1] = R(0.5) * (dp[0] + hdn_p * inv_c);
  } else {
    const R gm1 = R(P.gamma - 1.0);
    const R c = w.c;
    const R inv_c2 = R(1) / (c * c);
    const R q2 = R(0.5) * (w.u * w.u + w.v * w.v);
    const R un = dir == 0 ? w.u : w.v;
    const R ut = dir == 0 ? w.v : w.u;
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const R* dU = s == 0 ? dm : dp;
      R* out = s == 0 ? wm : wp;
      R dmy = D == 2 ? dU[2] : R(0);
      R chem = R(0);
      if constexpr (SYS == SYS_REACT) chem = R(P.q) * dU[D + 2];
      R dpres = gm1 * (dU[D + 1] - w.u * dU[1] - w.v * dmy + q2 * dU[0] - chem);
      R rdun = (dir == 0 ? dU[1] : dmy) - un * dU[0];  // rho d(u_n)
      out[0] = R(0.5) * (dpres - c * rdun) * inv_c2;
      out[1] = dU[0] - dpres * inv_c2;
      int r = 2;
      if constexpr (D == 2) {
        out[r++] = (dir == 0 ? dmy : dU[1]) - ut * dU[0];  // rho d(u_t)
      }
      if constexpr (SYS == SYS_REACT) out[r++] = dU[D + 2] - w.Y * dU[0];  // rho dY
      out[M - 1] = R(0.5) * (dpres + c * rdun) * inv_c2;
    }
  }
  R nu = R(0);
#pragma unroll
  for (int r = 0; r < M; r++) {
    R am = rabs(wm[r]), ap = rabs(wp[r]);
    nu += rabs(wp[r] - wm[r]) / (am + ap + dx) + am + ap;
  }
  return nu;
}

// Bed gradient of b = amp exp(-((x-xc)^2 + (y-yc)^2)/w2)
template <class R>
__device__ __forceinline__ void bed_gradient(const DevParams& P, double x, double y, int D, R* bx, R* by) {
  R dxr = R(x - P.bed_xc), dyr = D == 2 ? R(y - P.bed_yc) : R(0);
  R b = R(P.bed_amp) * rexp_(-(dxr * dxr + dyr * dyr) / R(P.bed_w2));
  *bx = R(-2.0) * dxr / R(P.bed_w2) * b;
  *by = R(-2.0) * dyr / R(P.bed_w2) * b;
}

// Arrhenius rate R = K rho Y exp(-Ti/T), T = p/rho (Section 5.4), in FP64
__device__ __forceinline__ double arrhenius(const DevParams& P, double rho, double momsq, double E, double z) {
  double pres = (P.gamma - 1.0) * (E - 0.5 * momsq / rho - P.q * z);
  return P.K * z * exp(-P.Ti / (pres / rho));
}

// Source S(U) at (x, y).  Shallow water: bed slope; reactive: Arrhenius
// (evaluated in FP64 in both precisions).
template <int SYS, int D, class R>
__device__ __forceinline__ void source(const DevParams& P, const R* U, double x, double y, R* S) {
  constexpr int M = Fields<SYS, D>::M;
#pragma unroll
  for (int c = 0; c < M; c++) S[c] = R(0);
  if constexpr (SYS == SYS_SWE) {
    if (P.bed_amp != 0.0) {
      R bx, by;
      bed_gradient<R>(P, x, y, D, &bx, &by);
      S[1] = -R(P.g) * U[0] * bx;
      if constexpr (D == 2) S[2] = -R(P.g) * U[0] * by;
    }
  } else if constexpr (SYS == SYS_REACT) {
    if (P.K != 0.0) {
      double rho = (double)U[0], m1 = (double)U[1], m2 = D == 2 ? (double)U[2] : 0.0;
      S[D + 2] = R(-arrhenius(P, rho, m1 * m1 + m2 * m2, (double)U[D + 1], (double)U[D + 2]));
    }
  }
}

// Eq. (2.8): U^{n+1} = Ubar + dt/2 S(U^{n+1}).  Shallow water: no mass source,
// so the momentum update is explicit in h^{n+1} = hbar.  Reactive: a scalar
// equation g(z) = z - zbar + dt/2 R(z) = 0 in z = rho*Y, solved in FP64 by
// Newton's method safeguarded by bisection on the bracket between 0 and zbar.
// Returns status bits.
template <int SYS, int D, class R>
__device__ __forceinline__ unsigned implicit_moment(const DevParams& P, const R* Ubar, double x, double y,
                                                    double dt, R* Un) {
  constexpr int M = Fields<SYS, D>::M;
#pragma unroll
  for (int c = 0; c < M; c++) Un[c] = Ubar[c];
  if constexpr (SYS == SYS_SWE) {
    if (P.bed_amp != 0.0) {
      R bx, by;
      bed_gradient<R>(P, x, y, D, &bx, &by);
      R half = R(0.5 * dt);
      Un[1] = Ubar[1] + half * (-R(P.g) * Un[0] * bx);
      if constexpr (D == 2) Un[2] = Ubar[2] + half * (-R(P.g) * Un[0] * by);
    }
    return 0u;
  } else if constexpr (SYS == SYS_REACT) {
    if (P.K == 0.0) return 0u;
    const double zbar = (double)Ubar[D + 2];
    if (zbar == 0.0) return 0u;
    const double rho = (double)Ubar[0], E = (double)Ubar[D + 1];
    const double m1 = (double)Ubar[1], m2 = D == 2 ? (double)Ubar[2] : 0.0;
    const double momsq = m1 * m1 + m2 * m2;
    const double hk = 0.5 * dt * P.K;
    const double dTdz = -(P.gamma - 1.0) * P.q / rho;
    const double e0 = (P.gamma - 1.0) * (E - 0.5 * momsq / rho) / rho;  // T at z = 0
    double lo = zbar < 0.0 ? zbar : 0.0, hi = zbar < 0.0 ? 0.0 : zbar;
    double z = zbar / (1.0 + hk * exp(-P.Ti / (e0 + dTdz * zbar)));
    unsigned st = ST_NOROOT;
    for (int it = 0; it < 60; it++) {
      double T = e0 + dTdz * z;
      double ex = exp(-P.Ti / T);
      double gz = z - zbar + hk * z * ex;
      if (gz == 0.0) { st = 0u; break; }
      if (gz > 0.0) hi = z; else lo = z;
      double dg = 1.0 + hk * ex * (1.0 + z * P.Ti / (T * T) * dTdz);
      double zn = z - gz / dg;
      if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
      double tol = 1e-15 * fmax(fabs(zbar), 1e-300);
      if (fabs(zn - z) <= tol) { z = zn; st = 0u; break; }
      z = zn;
    }
    Un[D + 2] = R(z);
    return st;
  } else {
    return 0u;
  }
}

// status bits of a new state U^{n+1}
template <int SYS, int D, class R>
__device__ __forceinline__ unsigned state_status(const DevParams& P, const R* U) {
  constexpr int M = Fields<SYS, D>::M;
  bool bad = false;
#pragma unroll
  for (int c = 0; c < M; c++) bad |= !(rabs(U[c]) <= R(3.0e38));  // NaN or inf
  unsigned st = 0u;
  if constexpr (SYS == SYS_EULER || SYS == SYS_REACT) {
    Prim<R> w = primitives<SYS, D, R>(P, U);
    bad |= !(w.rho > R(0)) || !(w.p > R(0));
  } else if constexpr (SYS == SYS_SWE) {
    if (U[0] < R(-1e-12)) st |= ST_NEGATIVE_DEPTH;
  }
  return st | (bad ? ST_NONPHYSICAL : 0u);
}

}  // namespace lbmh
