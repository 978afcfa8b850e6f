// Fused 3D (D3Q7) step: one kernel per step after the ghost layers of U.
//
// A block of 256 threads owns a tile of 32 x 8 output columns (x, y) and
// marches a chunk of planes along z.  The only state read from global memory
// besides the distributions is U^n on the ghost-extended grid (written as a
// side product by the previous step, its ghost layers refilled before this
// kernel); the indicator (Eq. 2.13/2.14), its 27-point box sum and omega
// (Eq. 2.15/2.16) are computed in shared memory as the tile marches, instead
// of round trips through global nu and omega arrays.  Per plane q:
//   U(q) on the tile + 3 arrives (cp.async, one plane ahead) in a ring of 4 planes
//   1  nu(q-1) on the tile + 2 from U(q-2..q)         (ring of 3 nu planes)
//   2  omega(q-2) on the tile + 1 from nu(q-3..q-1)
//   3  posts of plane q-2: every direction at the tile's own columns, the one
//      direction each halo column or row streams into the tile
//   4  plane q-3 streamed (F_k(x) = post_k(x - e_k), Eq. 2.2), the implicit
//      moment (2.8) and second half-source; f^{n+1} and U^{n+1} stored
// Sideways posts pass between lanes by warp shuffles (x) and shared memory (y,
// and the halo); the +-z posts stay in the thread's registers.  Every node's
// values are those of the four-kernel path (the same expressions in the same
// order), so the two paths agree to rounding.
#pragma once
#include "lbm3d.cuh"

namespace lbmh {

constexpr int kTX3 = 32, kTY3 = 8, kThreads3F = kTX3 * kTY3;
constexpr int kUW3 = kTX3 + 6, kUH3 = kTY3 + 6;  // U tile + 3
constexpr int kNW3 = kTX3 + 4, kNH3 = kTY3 + 4;  // nu tile + 2
constexpr int kOW3 = kTX3 + 2, kOH3 = kTY3 + 2;  // omega tile + 1
constexpr int kURing3 = 4;

template <int M, class R>
struct Smem3F {
  static constexpr size_t u_elems = (size_t)kURing3 * M * kUH3 * kUW3;
  static constexpr size_t nu_elems = (size_t)3 * kNH3 * kNW3;
  static constexpr size_t om_elems = (size_t)kOH3 * kOW3;
  static constexpr size_t py_elems = (size_t)M * (kTY3 + 1) * kTX3;  // post_{+y}, row ty at ty + 1
  static constexpr size_t my_elems = (size_t)M * (kTY3 + 1) * kTX3;  // post_{-y}, row ty at ty
  static constexpr size_t hx_elems = (size_t)2 * M * kTY3;           // halo columns' post_{+x} / post_{-x}
  static constexpr size_t total = (u_elems + nu_elems + om_elems + py_elems + my_elems + hx_elems) * sizeof(R);
};

template <class R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(R) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// resident blocks per SM the registers are budgeted for
template <int SYS, class R>
constexpr int k3f_min_blocks() { return sizeof(R) == 4 ? 2 : 1; }

template <int SYS, class R>
__global__ void __launch_bounds__(kThreads3F, k3f_min_blocks<SYS, R>())
    k3_fused(DevParams P, R* const* buf, Ctl* ctl, int slot, ExtGeom3 G, R* Ue2, double* partials, int zc) {
  constexpr int M = Fields3<SYS>::M, Q = 7;
  constexpr bool SRC = SYS == SYS_REACT;
  using L = Smem3F<M, R>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* Us = (R*)smem_raw;              // [ring][M][kUH3][kUW3]
  R* nus = Us + L::u_elems;          // [3][kNH3][kNW3]
  R* oms = nus + L::nu_elems;        // [kOH3][kOW3]
  R* pys = oms + L::om_elems;        // [M][kTY3 + 1][kTX3]
  R* mys = pys + L::py_elems;        // [M][kTY3 + 1][kTX3]
  R* hxs = mys + L::my_elems;        // [2][M][kTY3]
  __shared__ StepCoef3 s_cf;
  __shared__ R s_k[9];  // a0, 1/(2 lambda), dt/2, alpha_0..2, a_1..3
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  if (t == 0) {
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
  }
  __syncthreads();
  const StepCoef3 cf = s_cf;
  const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (!cf.active) {
    if (bid == 0 && t == 0) advance_ctl3(ctl, slot, cf);
    return;
  }
  const int par = ctl->parity[slot];
  const R* f = buf[par];
  R* fo = buf[par ^ 1];
  const R* Ue = ue_copy<M>(Ue2, G, par);
  R* Uo_ext = ue_copy<M>(Ue2, G, par ^ 1);  // U^{n+1} of the interior, for the next step
  const long long n = (long long)G.ex * G.ey * G.ez;
  const long long nf = 7ll * M * P.plane;
  unsigned int* const stc = &ctl->status;
  const Phys<R> K = make_phys<R>(P);
  const R a0 = s_k[0], inv2l = s_k[1], hdt = s_k[2];
  const R al[3] = {s_k[3], s_k[4], s_k[5]};
  const R aj[3] = {s_k[6], s_k[7], s_k[8]};
  const bool fixed_omega = P.omega_mode == 1;
  R om_fixed;
  if constexpr (sizeof(R) == 4)
    om_fixed = P.pf.omega_fixed;
  else
    om_fixed = P.omega_fixed;

  const int x0 = blockIdx.x * kTX3, y0 = blockIdx.y * kTY3;
  const int zb = blockIdx.z * zc, ze = min(zb + zc, P.nz3);
  const int x = x0 + tx, y = y0 + ty;
  const bool own_valid = x < P.nx && y < P.ny3;
  const int mx = map_index(x, P.nx, P.bc[0], P.bc[1]), my = map_index(y, P.ny3, P.bc[2], P.bc[3]);

  // U(plane) on the tile + 3 into ring slot plane % 4 (ext coordinates: x0 + ix,
  // y0 + iy, plane + GH; points past the extension are never used for an
  // output and are not copied)
  auto load_u = [&](int plane) {
    R* dst = Us + (size_t)(((plane % kURing3) + kURing3) % kURing3) * M * kUH3 * kUW3;
    const int ek = plane + GH;
    constexpr int items = M * kUH3 * kUW3;
    for (int it = t; it < items; it += kThreads3F) {
      const int c = it / (kUH3 * kUW3), rem = it % (kUH3 * kUW3), iy = rem / kUW3, ix = rem % kUW3;
      const int ei = x0 + ix, ej = y0 + iy;
      if (ei < G.ex && ej < G.ey) cp_async_elem(dst + it, Ue + chk((long long)c * n + G.idx(ek, ej, ei), (long long)M * n, stc));
    }
    cp_async_commit();
  };
  auto uslot = [&](int plane) -> const R* {
    return Us + (size_t)(((plane % kURing3) + kURing3) % kURing3) * M * kUH3 * kUW3;
  };

  R sp0 = R(0), sp1 = R(0), sp2 = R(0);
  Acc<R> acc[M];
#pragma unroll
  for (int c = 0; c < M; c++) acc[c].init();
  unsigned st = 0u;
  // registers carried between planes: the posts of plane q-3 streamed sideways
  // into the lane's column (and its own post_0), post_{+z} of planes q-3, q-4
  R kp0[M], kxp[M], kxm[M], kyp[M], kym[M], pz1[M], pz2[M];
#pragma unroll
  for (int c = 0; c < M; c++) kp0[c] = kxp[c] = kxm[c] = kyp[c] = kym[c] = pz1[c] = pz2[c] = R(0);

  const int q0 = zb - 3, q1 = ze + 2;
  load_u(q0);
#pragma unroll 1
  for (int q = q0; q <= q1; q++) {
    cp_async_wait_all();  // U(q) of this thread's copies
    if (q < q1) load_u(q + 1);
    __syncthreads();      // U(q) of every thread visible
    // 1: nu(q - 1) on the tile + 2
    if (q >= zb - 1) {
      const R* Um1 = uslot(q - 2);
      const R* U00 = uslot(q - 1);
      const R* Up1 = uslot(q);
      R* nd = nus + (size_t)(((q - 1) % 3 + 3) % 3) * kNH3 * kNW3;
      for (int it = t; it < kNH3 * kNW3; it += kThreads3F) {
        const int iy = it / kNW3, ix = it % kNW3;
        const int o = (iy + 1) * kUW3 + (ix + 1);  // position in the U tile
        constexpr int CS = kUH3 * kUW3;
        R U0[M], dm[M], dp[M];
#pragma unroll
        for (int c = 0; c < M; c++) U0[c] = U00[c * CS + o];
        const Prim3<R> w = prim3<SYS, R>(K, U0);
        R sum = R(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
          for (int c = 0; c < M; c++) {
            const R um = d == 0 ? U00[c * CS + o - 1] : (d == 1 ? U00[c * CS + o - kUW3] : Um1[c * CS + o]);
            const R up = d == 0 ? U00[c * CS + o + 1] : (d == 1 ? U00[c * CS + o + kUW3] : Up1[c * CS + o]);
            dm[c] = U0[c] - um;
            dp[c] = up - U0[c];
          }
          sum += theta3<SYS, R>(K, w, d, dm, dp);
        }
        nd[it] = sum;
      }
    }
    __syncthreads();
    // 2: omega(q - 2) on the tile + 1 (27 terms in the order (bk, bj, bi))
    if (q >= zb + 1) {
      const R* nb[3];
#pragma unroll
      for (int pz = 0; pz < 3; pz++) nb[pz] = nus + (size_t)(((q - 3 + pz) % 3 + 3) % 3) * kNH3 * kNW3;
      for (int it = t; it < kOH3 * kOW3; it += kThreads3F) {
        const int jy = it / kOW3, jx = it % kOW3;
        R w;
        if (fixed_omega) {
          w = om_fixed;
        } else {
          R s = R(0);
#pragma unroll
          for (int pz = 0; pz < 3; pz++)
#pragma unroll
            for (int bj = 0; bj < 3; bj++)
#pragma unroll
              for (int bi = 0; bi < 3; bi++) s += nb[pz][(jy + bj) * kNW3 + jx + bi];
          w = R(1) + fdiv(R(1), R(1) + s);
        }
        oms[it] = w;
      }
    }
    __syncthreads();
    if (q >= zb + 1) {
      // 3: posts of plane pp = q - 2
      const int pp = q - 2;
      const int mk = map_index(pp, P.nz3, P.bc_z[0], P.bc_z[1]);
      const R* Ut = uslot(pp);
      constexpr int CS = kUH3 * kUW3;
      // own column: all seven directions
      R pown[Q][M];
      {
        R U[M], fq[Q][M], S[M], F[3][M];
        const int o = (ty + 3) * kUW3 + (tx + 3);
#pragma unroll
        for (int c = 0; c < M; c++) U[c] = Ut[c * CS + o];
        const R w = oms[(ty + 1) * kOW3 + (tx + 1)];
        const long long off = cell3(P, mx, my, mk);
#pragma unroll
        for (int k = 0; k < Q; k++)
#pragma unroll
          for (int c = 0; c < M; c++) fq[k][c] = f[chk((long long)(k * M + c) * P.plane + off, nf, stc)];
        const Prim3<R> pw = prim3<SYS, R>(K, U);
        if constexpr (SRC)
          source3<SYS, R>(K, U, S);
        else
#pragma unroll
          for (int c = 0; c < M; c++) S[c] = R(0);
#pragma unroll
        for (int d = 0; d < 3; d++) flux3<SYS, R>(K, P, U, pw, d, F[d]);
#pragma unroll
        for (int c = 0; c < M; c++) {
          R v = fq[0][c] - w * (fq[0][c] - a0 * U[c]);
          if constexpr (SRC) v += hdt * a0 * S[c];
          pown[0][c] = v;
        }
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
          for (int c = 0; c < M; c++) {
            const R fp = (al[d] * U[c] + F[d][c]) * inv2l, fm = (al[d] * U[c] - F[d][c]) * inv2l;
            R vp = fq[1 + d][c] - w * (fq[1 + d][c] - fp);
            R vm = fq[4 + d][c] - w * (fq[4 + d][c] - fm);
            if constexpr (SRC) {
              vp += hdt * aj[d] * S[c];
              vm += hdt * aj[d] * S[c];
            }
            pown[1 + d][c] = vp;
            pown[4 + d][c] = vm;
          }
      }
#pragma unroll
      for (int c = 0; c < M; c++) {
        pys[(c * (kTY3 + 1) + ty + 1) * kTX3 + tx] = pown[2][c];
        mys[(c * (kTY3 + 1) + ty) * kTX3 + tx] = pown[5][c];
      }
      // halo: the one direction each halo column / row streams into the tile
      if (t < 2 * kTY3 + 2 * kTX3) {
        int hx, hy, qq, dir;
        if (t < kTY3) { hx = -1; hy = t; qq = 1; dir = 0; }
        else if (t < 2 * kTY3) { hx = kTX3; hy = t - kTY3; qq = 4; dir = 0; }
        else if (t < 2 * kTY3 + kTX3) { hx = t - 2 * kTY3; hy = -1; qq = 2; dir = 1; }
        else { hx = t - 2 * kTY3 - kTX3; hy = kTY3; qq = 5; dir = 1; }
        const int gxh = x0 + hx, gyh = y0 + hy;
        const int o = (hy + 3) * kUW3 + (hx + 3);
        R U[M], fq[M], S[M], F[M];
#pragma unroll
        for (int c = 0; c < M; c++) U[c] = Ut[c * CS + o];
        const R w = oms[(hy + 1) * kOW3 + (hx + 1)];
        const long long off = cell3(P, map_index(gxh, P.nx, P.bc[0], P.bc[1]), map_index(gyh, P.ny3, P.bc[2], P.bc[3]), mk);
#pragma unroll
        for (int c = 0; c < M; c++) fq[c] = f[chk((long long)(qq * M + c) * P.plane + off, nf, stc)];
        const Prim3<R> pw = prim3<SYS, R>(K, U);
        if constexpr (SRC)
          source3<SYS, R>(K, U, S);
        else
#pragma unroll
          for (int c = 0; c < M; c++) S[c] = R(0);
        flux3<SYS, R>(K, P, U, pw, dir, F);
        R* dst = qq == 1 ? hxs + hy : (qq == 4 ? hxs + M * kTY3 + hy
                                              : (qq == 2 ? pys + hx : mys + kTY3 * kTX3 + hx));
        const int cstride = (qq == 1 || qq == 4) ? kTY3 : (kTY3 + 1) * kTX3;
#pragma unroll
        for (int c = 0; c < M; c++) {
          const R feq = qq <= 3 ? (al[dir] * U[c] + F[c]) * inv2l : (al[dir] * U[c] - F[c]) * inv2l;
          R v = fq[c] - w * (fq[c] - feq);
          if constexpr (SRC) v += hdt * aj[dir] * S[c];
          dst[c * cstride] = v;
        }
      }
      // 4: stream plane p = q - 3 into the lane's column
      const int p = q - 3;
      if (p >= zb && own_valid) {
        R Fk[Q][M];
#pragma unroll
        for (int c = 0; c < M; c++) {
          Fk[0][c] = kp0[c];
          Fk[1][c] = kxp[c];
          Fk[2][c] = kyp[c];
          Fk[3][c] = pz2[c];         // post_{+z} of plane p - 1
          Fk[4][c] = kxm[c];
          Fk[5][c] = kym[c];
          Fk[6][c] = pown[6][c];     // post_{-z} of plane p + 1
        }
        R Ubar[M];
#pragma unroll
        for (int c = 0; c < M; c++) {
          R sum = R(0);
#pragma unroll
          for (int k = 0; k < Q; k++) sum += Fk[k][c];
          Ubar[c] = sum;
        }
        R Sn[M];
#pragma unroll
        for (int c = 0; c < M; c++) Sn[c] = R(0);
        if constexpr (SRC) {
          if (K.react && Ubar[5] != R(0)) {
            R Un[M];
#pragma unroll
            for (int c = 0; c < M; c++) Un[c] = Ubar[c];
            st |= react_implicit3<R>(K, Ubar, cf.dt, hdt, &Un[5]);
            source3<SYS, R>(K, Un, Sn);
          }
        }
        const long long oo = cell3(P, x, y, p);
        R Uo[M];
#pragma unroll
        for (int c = 0; c < M; c++) Uo[c] = R(0);
#pragma unroll
        for (int k = 0; k < Q; k++) {
          const R akq = k == 0 ? a0 : aj[(k - 1) % 3];
#pragma unroll
          for (int c = 0; c < M; c++) {
            R v = Fk[k][c];
            if constexpr (SRC) v += hdt * akq * Sn[c];
            fo[chk((long long)(k * M + c) * P.plane + oo, nf, stc)] = v;
            Uo[c] += v;
          }
        }
        const long long eo = G.idx(p + GH, y + GH, x + GH);
#pragma unroll
        for (int c = 0; c < M; c++) Uo_ext[chk((long long)c * n + eo, (long long)M * n, stc)] = Uo[c];
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
      __syncthreads();  // the sideways posts of plane q - 2 are in shared memory
      // gather them for plane q - 2 (streamed one plane later)
#pragma unroll
      for (int c = 0; c < M; c++) {
        const R left = __shfl_up_sync(0xffffffffu, pown[1][c], 1);
        const R right = __shfl_down_sync(0xffffffffu, pown[4][c], 1);
        kxp[c] = tx == 0 ? hxs[c * kTY3 + ty] : left;
        kxm[c] = tx == 31 ? hxs[(M + c) * kTY3 + ty] : right;
        kyp[c] = pys[(c * (kTY3 + 1) + ty) * kTX3 + tx];
        kym[c] = mys[(c * (kTY3 + 1) + ty + 1) * kTX3 + tx];
        kp0[c] = pown[0][c];
        pz2[c] = pz1[c];
        pz1[c] = pown[3][c];
      }
    }
  }
  // side outputs per warp (partial slot bid * 8 + warp): no block barrier
  warp_side_outputs3<M, R>(sp0, sp1, sp2, acc, ctl, (slot + 1) % 3,
                           partials + (bid * (kThreads3F / 32) + ty) * M, st);
  if (bid == 0 && t == 0) advance_ctl3(ctl, slot, cf);
}

// launch shape of the fused 3D step: tiles of 32 x 8 columns, chunks of zc planes
inline dim3 grid3_fused(int nx, int ny, int nz, int zc) {
  return dim3((unsigned)((nx + kTX3 - 1) / kTX3), (unsigned)((ny + kTY3 - 1) / kTY3), (unsigned)((nz + zc - 1) / zc));
}

}  // namespace lbmh
