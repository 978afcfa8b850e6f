// Per-node physics of the four systems on the hot path, templated on the
// system, the dimension and the arithmetic type R (float or double):
// flux F_j(U), the speed bound max_r |lambda_r(dF_j/dU)|, the characteristic
// smoothness indicator, the source S(U) and the implicit moment of Eq. (2.8).
//
// All constants arrive pre-converted to R in a Phys<R> block built once per
// thread, so the FP32 path issues no FP64 instruction per node; its Arrhenius
// root falls back to FP64 only where the FP32 Newton iteration does not
// converge.
#pragma once
#include "common.cuh"

namespace lbmh {

__device__ __forceinline__ float rabs(float x) { return fabsf(x); }
__device__ __forceinline__ double rabs(double x) { return fabs(x); }

// Division, reciprocal and square root: IEEE in FP64; in FP32 the MUFU
// approximations (<= 2 ulp), which is the precision the FP32 mode runs at.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float frcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double frcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float fsqrt(float x) {
  // x * rsqrt(x) with the argument of rsqrt kept positive: 0 stays 0; a
  // negative x (a non-physical state, flagged separately) gives a negative c
  return x * rsqrtf(fmaxf(x, 1e-37f));
}
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }

// The coefficient a_0 = 1 - sum_j alpha_j / lambda of the rest equilibrium
// (Eq. 2.20) in FP32, as an unevaluated sum hi + lo of two floats built from
// the FP32-rounded alpha_j and 1/(2 lambda) that the moving equilibria use, so
// that a_0 + sum_j 2 alpha_j / (2 lambda) = 1 holds to ~2^-48.  Rounded on
// their own, the FP32 coefficients made a node's equilibria sum to U (1 + d)
// with one d ~ 2^-25 for every node of a step, and each step moved the mass by
// omega d: a drift linear in the number of steps (1D Shu-Osher, 2^18 nodes,
// 756,609 steps: L1 1.6e-2 against FP64; with hi + lo 8.5e-4).  In FP64 hi is
// a_0 and lo is 0.  `al` holds the d FP32 alpha_j.
template <class R>
struct RestCoef {
  R hi, lo;
};
template <class R>
__device__ __forceinline__ RestCoef<R> rest_coef(double a0, const R* al, int d, R inv2l) {
  RestCoef<R> c;
  if constexpr (sizeof(R) == 4) {
    // 1 - sum_j 2 al_j inv2l in FP32 arithmetic without FP64 (a dependent
    // FP64 chain at the start of each block cost the 1D step ~3 %): every
    // product split exactly as p + e (fma), the running sum hi + lo kept by
    // TwoSum; 2 p and 2 e are exact
    float hi = 1.0f, lo = 0.0f;
    for (int j = 0; j < d; j++) {
      const float p = al[j] * inv2l;
      const float e = fmaf(al[j], inv2l, -p);  // al_j inv2l = p + e exactly
      const float b = -2.0f * p;
      const float s2 = hi + b, bb = s2 - hi;
      lo += ((hi - (s2 - bb)) + (b - bb)) - 2.0f * e;
      hi = s2;
    }
    const float t = hi + lo;
    c.lo = lo - (t - hi);
    c.hi = t;
  } else {
    c.hi = R(a0);
    c.lo = R(0);
  }
  return c;
}

// the rest equilibrium a_0 U with a_0 = hi + lo (FP32) or hi (FP64)
template <class R>
__device__ __forceinline__ R rest_eq(R hi, R lo, R U) {
  if constexpr (sizeof(R) == 4)
    return hi * U + lo * U;
  else
    return hi * U;
}

// Problem constants in the arithmetic type of the path.
template <class R>
struct Phys {
  R gamma, gm1, g, half_g, h_dry, cmin, q, adv0, adv1, dx;
  R bed_amp, bed_inv_w2, bed_m2_inv_w2;  // amp, 1/w2, -2/w2
  R xb, yb;                              // x0 + dx/2 - xc, y0 + dx/2 - yc: node i sits at xb + i dx
  double gamma_d, q_d, K, Ti;            // Arrhenius, FP64
  R Kr, Tir;                             // Arrhenius in the path's precision
  bool bed, react;
};

template <class R>
__device__ __forceinline__ Phys<R> make_phys(const DevParams& P) {
  Phys<R> k;
  if constexpr (sizeof(R) == 4) {  // the host-rounded FP32 constants
    const PhysConstF& f = P.pf;
    k.gamma = f.gamma;
    k.gm1 = f.gm1;
    k.g = f.g;
    k.half_g = f.half_g;
    k.h_dry = f.h_dry;
    k.cmin = f.cmin;
    k.q = f.q;
    k.adv0 = f.adv0;
    k.adv1 = f.adv1;
    k.dx = f.dx;
    k.bed_amp = f.bed_amp;
    k.bed_inv_w2 = f.bed_inv_w2;
    k.bed_m2_inv_w2 = f.bed_m2_inv_w2;
    k.xb = f.xb;
    k.yb = f.yb;
    k.Kr = f.K;
    k.Tir = f.Ti;
  } else {
    k.gamma = P.gamma;
    k.gm1 = P.gamma - 1.0;
    k.g = P.g;
    k.half_g = 0.5 * P.g;
    k.h_dry = P.h_dry;
    k.cmin = sqrt(P.g * P.h_dry);
    k.q = P.q;
    k.adv0 = P.adv[0];
    k.adv1 = P.adv[1];
    k.dx = P.dx;
    k.bed_amp = P.bed_amp;
    k.bed_inv_w2 = 1.0 / P.bed_w2;
    k.bed_m2_inv_w2 = -2.0 / P.bed_w2;
    k.xb = P.x0 + 0.5 * P.dx - P.bed_xc;
    k.yb = P.y0 + 0.5 * P.dx - P.bed_yc;
    k.Kr = P.K;
    k.Tir = P.Ti;
  }
  k.gamma_d = P.gamma;
  k.q_d = P.q;
  k.K = P.K;
  k.Ti = P.Ti;
  k.bed = P.has_bed != 0;
  k.react = P.has_react != 0;
  return k;
}

template <int SYS>
struct HasSource {
  static constexpr bool value = SYS == SYS_SWE || SYS == SYS_REACT;
};

// Primitive variables of an Euler-type or shallow-water state.
template <class R>
struct Prim {
  R rho, u, v, p, c, Y;  // Euler / reactive; for shallow water rho holds h
};

template <int SYS, int D, class R>
__device__ __forceinline__ Prim<R> primitives(const Phys<R>& K, const R* U) {
  Prim<R> w;
  w.Y = R(0);
  w.p = R(0);
  if constexpr (SYS == SYS_EULER || SYS == SYS_REACT) {
    w.rho = U[0];
    R inv = frcp(w.rho);
    w.u = U[1] * inv;
    w.v = D == 2 ? U[2] * inv : R(0);
    R kin = R(0.5) * w.rho * (w.u * w.u + w.v * w.v);
    R chem = R(0);
    if constexpr (SYS == SYS_REACT) {
      w.Y = U[D + 2] * inv;
      chem = K.q * U[D + 2];
    }
    w.p = K.gm1 * (U[D + 1] - kin - chem);
    w.c = fsqrt(K.gamma * w.p * inv);
  } else if constexpr (SYS == SYS_SWE) {
    w.rho = U[0];
    if (w.rho < K.h_dry) {  // dry node: at rest
      w.u = R(0);
      w.v = R(0);
    } else {
      R inv = frcp(w.rho);
      w.u = U[1] * inv;
      w.v = D == 2 ? U[2] * inv : R(0);
    }
    w.c = fsqrt(K.g * (w.rho > R(0) ? w.rho : R(0)));
  } else {
    w.rho = w.u = w.v = w.c = R(0);
  }
  return w;
}

// Flux F_dir(U): Section 5 (shallow water, reactive Euler; Euler is the
// reactive flux without species).
template <int SYS, int D, class R>
__device__ __forceinline__ void flux(const Phys<R>& K, const R* U, const Prim<R>& w, int dir, R* F) {
  if constexpr (SYS == SYS_ADV) {
    F[0] = (dir == 0 ? K.adv0 : K.adv1) * U[0];
  } else if constexpr (SYS == SYS_SWE) {
    R vn = dir == 0 ? w.u : w.v;
    R pres = K.half_g * w.rho * w.rho;
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
__device__ __forceinline__ R max_speed(const Phys<R>& K, const Prim<R>& w, int dir) {
  if constexpr (SYS == SYS_ADV) {
    return rabs(dir == 0 ? K.adv0 : K.adv1);
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
__device__ __forceinline__ R theta_sum(const Phys<R>& K, const Prim<R>& w, int dir, const R* dm, const R* dp) {
  constexpr int M = Fields<SYS, D>::M;
  R wm[M], wp[M];
  if constexpr (SYS == SYS_ADV) {
    wm[0] = dm[0];
    wp[0] = dp[0];
  } else if constexpr (SYS == SYS_SWE) {
    R c = w.c < K.cmin ? K.cmin : w.c;
    R inv_c = frcp(c);
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
    const R c = w.c;
    const R inv_c2 = frcp(c * c);
    const R q2 = R(0.5) * (w.u * w.u + w.v * w.v);
    const R un = dir == 0 ? w.u : w.v;
    const R ut = dir == 0 ? w.v : w.u;
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const R* dU = s == 0 ? dm : dp;
      R* out = s == 0 ? wm : wp;
      R dmy = D == 2 ? dU[2] : R(0);
      R chem = R(0);
      if constexpr (SYS == SYS_REACT) chem = K.q * dU[D + 2];
      R dpres = K.gm1 * (dU[D + 1] - w.u * dU[1] - w.v * dmy + q2 * dU[0] - chem);
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
    nu += fdiv(rabs(wp[r] - wm[r]), am + ap + K.dx) + am + ap;
  }
  return nu;
}

// Gradient of the bed b = amp exp(-(xr^2 + yr^2)/w2); xr, yr relative to the
// bump centre
template <class R>
__device__ __forceinline__ void bed_gradient(const Phys<R>& K, R xr, R yr, R* bx, R* by) {
  R b = K.bed_amp * fexp(-(xr * xr + yr * yr) * K.bed_inv_w2);
  *bx = K.bed_m2_inv_w2 * xr * b;
  *by = K.bed_m2_inv_w2 * yr * b;
}

// Arrhenius rate R = K rho Y exp(-Ti/T), T = p/rho (Section 5.4), in FP64
template <class R>
__device__ __forceinline__ double arrhenius(const Phys<R>& K, double rho, double momsq, double E, double z) {
  double pres = (K.gamma_d - 1.0) * (E - 0.5 * momsq / rho - K.q_d * z);
  return K.K * z * exp(-K.Ti / (pres / rho));
}

// The same rate in FP32: T = p/rho, exp(-Ti rho / p) with the accurate expf
// (the FP32 mode's explicit half-source; its relative error is that of the
// FP32 state it is computed from)
__device__ __forceinline__ float arrhenius_f32(const Phys<float>& K, float rho, float momsq, float E, float z) {
  float pres = K.gm1 * (E - 0.5f * fdiv(momsq, rho) - K.q * z);
  return K.Kr * z * expf(-fdiv(K.Tir * rho, pres));
}

// Fields to which the half-source terms dt/2 a_k S_c are added.  Reactive
// Euler: rho*Y alone (S is identically 0 in the other fields, and adding
// dt/2 a_k * 0 would still cost a multiply-add per direction and field).  The
// other systems add to every field: for shallow water, skipping the zero field
// together with taking the second half-source dt/2 S(U^{n+1}) as U^{n+1} - Ubar
// (Eq. 2.8; the kernels' moment step does so for reactive Euler) made the 2D
// step slower (2048^2 dam break 0.1545 against 0.150 ms).
template <int SYS, int D>
__host__ __device__ constexpr bool src_field(int c) {
  return SYS == SYS_REACT ? c == D + 2 : true;
}

// Source S(U) at a node whose position relative to the bump centre is
// (xr, yr).  Shallow water: bed slope; reactive: Arrhenius (FP64 in the FP64
// mode, FP32 in the FP32 mode).
template <int SYS, int D, class R>
__device__ __forceinline__ void source(const Phys<R>& K, const R* U, R xr, R yr, R* S) {
  constexpr int M = Fields<SYS, D>::M;
#pragma unroll
  for (int c = 0; c < M; c++) S[c] = R(0);
  if constexpr (SYS == SYS_SWE) {
    if (K.bed) {
      R bx, by;
      bed_gradient<R>(K, xr, D == 2 ? yr : R(0), &bx, &by);
      S[1] = -K.g * U[0] * bx;
      if constexpr (D == 2) S[2] = -K.g * U[0] * by;
    }
  } else if constexpr (SYS == SYS_REACT) {
    if (K.react) {
      if constexpr (sizeof(R) == 4) {
        const float m2 = D == 2 ? U[2] : 0.0f;
        S[D + 2] = -arrhenius_f32(K, U[0], U[1] * U[1] + m2 * m2, U[D + 1], U[D + 2]);
      } else {
        double rho = (double)U[0], m1 = (double)U[1], m2 = D == 2 ? (double)U[2] : 0.0;
        S[D + 2] = R(-arrhenius(K, rho, m1 * m1 + m2 * m2, (double)U[D + 1], (double)U[D + 2]));
      }
    }
  }
}

// FP32 root of g(z) = z - zbar + dt/2 K z exp(-Ti/T(z)) (see implicit_moment):
// the same safeguarded Newton iteration in FP32, stopped when the Newton step
// falls below max(2^-22 |zbar|, 2^-126) (about two FP32 ulps of zbar, or the
// smallest normal float; the iterate is then rounded to FP32 storage anyway).  Returns 0 (converged), 1 (no convergence
// in 30 iterations: the caller solves in FP64) or 2 (non-finite state: no
// root is sought).
template <int D>
__device__ __forceinline__ int react_root_f32(const Phys<float>& K, const float* Ubar, float hdt, float* zout) {
  const float zbar = Ubar[D + 2], rho = Ubar[0], E = Ubar[D + 1];
  const float m2 = D >= 2 ? Ubar[2] : 0.0f;
  float momsq = Ubar[1] * Ubar[1] + m2 * m2;
  if constexpr (D == 3) momsq += Ubar[3] * Ubar[3];
  const float irho = frcp(rho);
  const float hk = hdt * K.Kr;  // dt/2 K
  const float dTdz = -K.gm1 * K.q * irho;
  const float e0 = K.gm1 * (E - 0.5f * momsq * irho) * irho;
  float lo = zbar < 0.0f ? zbar : 0.0f, hi = zbar < 0.0f ? 0.0f : zbar;
  float z = fdiv(zbar, 1.0f + hk * expf(-fdiv(K.Tir, e0 + dTdz * zbar)));
  if (!(fabsf(z) <= 3.0e38f)) return 2;
  // two FP32 ulps of zbar, but no less than the smallest normal float: once
  // zbar is subnormal (a burnt region decays geometrically towards 0) the
  // relative step underflows, the iteration alternates between neighbouring
  // subnormals, and only the absolute floor ends it (an error < 2^-126 in z)
  const float tol = fmaxf(0x1p-22f * fabsf(zbar), 0x1p-126f);
  for (int it = 0; it < 30; it++) {
    const float T = e0 + dTdz * z;
    const float a = fdiv(K.Tir, T);
    const float ex = expf(-a);
    const float gz = z - zbar + hk * z * ex;
    if (gz == 0.0f) {
      *zout = z;
      return 0;
    }
    if (gz > 0.0f) hi = z; else lo = z;
    const float dg = 1.0f + hk * ex * (1.0f + z * fdiv(a, T) * dTdz);
    float zn = z - fdiv(gz, dg);
    if (fabsf(zn - z) <= tol) {
      *zout = zn;
      return 0;
    }
    if (!(zn > lo && zn < hi)) zn = 0.5f * (lo + hi);
    z = zn;
  }
  return 1;
}

struct RootF64 {
  double z;
  unsigned st;
};

// FP64 root of g(z) = z - zbar + hk z exp(-Ti/T(z)), T(z) = e0 + dTdz z,
// hk = dt/2 K (see implicit_moment): Newton from the frozen-temperature guess,
// safeguarded by bisection on the bracket between 0 and zbar, until the step
// is below max(1e-15 |zbar|, 2^-1022).  A non-finite state returns z = zbar with ST_NOROOT.
__device__ __forceinline__ RootF64 react_root_f64(double rho, double momsq, double E, double zbar, double hk,
                                                  double gm1, double q, double Ti) {
  const double dTdz = -gm1 * q / rho;
  const double e0 = gm1 * (E - 0.5 * momsq / rho) / rho;  // T at z = 0
  double lo = zbar < 0.0 ? zbar : 0.0, hi = zbar < 0.0 ? 0.0 : zbar;
  double z = zbar / (1.0 + hk * exp(-Ti / (e0 + dTdz * zbar)));
  if (z != z) return RootF64{zbar, ST_NOROOT};
  for (int it = 0; it < 60; it++) {
    double T = e0 + dTdz * z;
    double ex = exp(-Ti / T);
    double gz = z - zbar + hk * z * ex;
    if (gz == 0.0) return RootF64{z, 0u};
    if (gz > 0.0) hi = z; else lo = z;
    double dg = 1.0 + hk * ex * (1.0 + z * Ti / (T * T) * dTdz);
    double zn = z - gz / dg;
    // converged when the Newton step is below the tolerance; tested before
    // the bracket guard, since z itself has just become a bracket end and a
    // sub-resolution step lands on it
    // (the absolute floor, the smallest normal double, ends the iteration
    // for a subnormal zbar as in the FP32 root)
    if (fabs(zn - z) <= fmax(1e-15 * fabs(zbar), 0x1p-1022)) return RootF64{zn, 0u};
    if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
    z = zn;
  }
  return RootF64{z, ST_NOROOT};
}

// The FP32 mode's fallback, out of line so that none of its FP64 work is
// scheduled into the FP32 path.
static __device__ __noinline__ RootF64 react_root_f64_fallback(float rho, float m1, float m2, float E, float zbar, double dt,
                                                               double Kc, double gamma, double q, double Ti) {
  const double d1 = (double)m1, d2 = (double)m2;
  return react_root_f64((double)rho, d1 * d1 + d2 * d2, (double)E, (double)zbar, 0.5 * dt * Kc, gamma - 1.0, q, Ti);
}

// Eq. (2.8): U^{n+1} = Ubar + dt/2 S(U^{n+1}).  Shallow water: no mass source,
// so the momentum update is explicit in h^{n+1} = hbar.  Reactive: a scalar
// equation g(z) = z - zbar + dt/2 R(z) = 0 in z = rho*Y, solved by Newton's
// method safeguarded by bisection on the bracket between 0 and zbar, from the
// frozen-temperature guess: in FP64 in the FP64 mode; in the FP32 mode in FP32
// first, in FP64 where the FP32 iteration does not converge.  Returns status
// bits.
template <int SYS, int D, class R>
__device__ __forceinline__ unsigned implicit_moment(const Phys<R>& K, const R* Ubar, R xr, R yr, double dt, R hdt,
                                                    R* Un) {
  constexpr int M = Fields<SYS, D>::M;
#pragma unroll
  for (int c = 0; c < M; c++) Un[c] = Ubar[c];
  if constexpr (SYS == SYS_SWE) {
    if (K.bed) {
      R bx, by;
      bed_gradient<R>(K, xr, D == 2 ? yr : R(0), &bx, &by);
      Un[1] = Ubar[1] + hdt * (-K.g * Un[0] * bx);
      if constexpr (D == 2) Un[2] = Ubar[2] + hdt * (-K.g * Un[0] * by);
    }
    return 0u;
  } else if constexpr (SYS == SYS_REACT) {
    if (!K.react) return 0u;
    if (Ubar[D + 2] == R(0)) return 0u;
    if constexpr (sizeof(R) == 4) {
      float zf;
      const int rc = react_root_f32<D>(K, Ubar, hdt, &zf);
      if (rc == 0) {
        Un[D + 2] = zf;
        return 0u;
      }
      if (rc == 2) return ST_NOROOT;  // z = zbar, as the FP64 path leaves it
    }
    RootF64 rt;
    if constexpr (sizeof(R) == 4) {
      rt = react_root_f64_fallback(Ubar[0], Ubar[1], D == 2 ? Ubar[2] : 0.0f, Ubar[D + 1], Ubar[D + 2], dt, K.K,
                                   K.gamma_d, K.q_d, K.Ti);
    } else {
      const double m1 = (double)Ubar[1], m2 = D == 2 ? (double)Ubar[2] : 0.0;
      rt = react_root_f64((double)Ubar[0], m1 * m1 + m2 * m2, (double)Ubar[D + 1], (double)Ubar[D + 2],
                          0.5 * dt * K.K, K.gamma_d - 1.0, K.q_d, K.Ti);
    }
    Un[D + 2] = R(rt.z);
    return rt.st;
  } else {
    return 0u;
  }
}

// status bits of a new state U^{n+1} with primitives w
template <int SYS, int D, class R>
__device__ __forceinline__ unsigned state_status(const R* U, const Prim<R>& w) {
  constexpr int M = Fields<SYS, D>::M;
  if constexpr (SYS == SYS_EULER || SYS == SYS_REACT) {
    // a NaN or inf in any field makes p NaN or +-inf (or rho non-positive)
    bool ok = w.rho > R(0) && w.p > R(0) && w.p <= R(3.0e38);
    return ok ? 0u : ST_NONPHYSICAL;
  } else {
    bool bad = false;
#pragma unroll
    for (int c = 0; c < M; c++) bad |= !(rabs(U[c]) <= R(3.0e38));  // NaN or inf
    unsigned st = bad ? ST_NONPHYSICAL : 0u;
    if constexpr (SYS == SYS_SWE) {
      if (U[0] < R(-1e-12)) st |= ST_NEGATIVE_DEPTH;
    }
    return st;
  }
}

// Error-free accumulation of FP32 values (Knuth's TwoSum into a hi/lo pair):
// the pair carries the running sum to ~2^-48 relative, so per-thread partial
// sums keep FP64-level accuracy without FP64 instructions per node.
template <class R>
struct Acc {
  R hi, lo;
  __device__ __forceinline__ void init() { hi = lo = R(0); }
  __device__ __forceinline__ void add(R x) {
    R s = hi + x;
    R bp = s - hi;
    R err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <>
struct Acc<double> {
  double hi;
  __device__ __forceinline__ void init() { hi = 0.0; }
  __device__ __forceinline__ void add(double x) { hi += x; }
  __device__ __forceinline__ double value() const { return hi; }
};

}  // namespace lbmh
