// Fused 3D (D3Q7) step: one kernel per step after the ghost layers of U.
//
// A block of 32 x TY threads owns a tile of 32 x TY output columns (x, y) and
// marches a chunk of planes along z (TY = 8, Tile3F).  The only state read
// from global memory besides the distributions is U^n on the ghost-extended
// grid (written as a side product by the previous step, its ghost layers
// refilled before this kernel); the indicator (Eq. 2.13/2.14), its 27-point
// box sum and omega (Eq. 2.15/2.16) are computed on chip as the tile marches,
// instead of round trips through global nu and omega arrays.  Per plane q:
//   U(q) on the tile + 3 arrives (one TMA box, one plane ahead) in a ring of 4
//   1  nu(q-1) on the tile + 2 from U(q-2..q); the thread that computes a
//      position keeps its nu of planes q-3, q-2 in registers and writes the
//      sum nu(q-3) + nu(q-2) + nu(q-1) there (one shared plane)
//   2  omega(q-2) on the tile + 1 from that plane's 3 x 3 window, by the thread
//      whose post needs it (own column, or the halo node it streams from)
//   3  posts of plane q-2: every direction at the tile's own columns, the one
//      direction each halo column or row streams into the tile
//   4  plane q-3 streamed (F_k(x) = post_k(x - e_k), Eq. 2.2), the implicit
//      moment (2.8) and second half-source; f^{n+1} and U^{n+1} stored
// The own columns' f^n of plane q-2 (all 7 m planes of the tile, one TMA box
// in FP32) is requested once plane q-3's posts are formed, so it lands while
// phases 1 and 2 of the next plane run (lanes of a ragged tile past the
// lattice's edge hold ghost nodes: they load the mapped node's f^n instead);
// the halo nodes' f^n (one direction each) is copied with cp.async at the
// start of the plane.  Sideways posts pass between lanes by warp shuffles (x)
// and shared memory (y, and the halo); the +-z posts stay in the thread's
// registers.  Every node's values
// are those of the four-kernel path (the same expressions in the same order),
// so the two paths agree to rounding.
#pragma once
#include "lbm3d.cuh"

namespace lbmh {

constexpr int kTX3 = 32;
constexpr int kUW3 = kTX3 + 8;  // U tile + 3 (38 columns used), loaded as a 40-column box
constexpr int kNW3 = kTX3 + 4;  // nu tile + 2
constexpr int kURing3 = 4;

// Tile height (rows of 32 columns; one warp per row).  8 rows, 256 threads.
// Tiles of 16 rows (512 threads, one block per SM) cut the indicator's
// recompute on the tile + 2 from 1.69 to 1.41 evaluations per output node,
// but ran slower (256^3 Euler FP32: 1.37 against 1.30 ms per step): two
// blocks of 8 warps overlap one another's barriers, one block of 16 does not.
template <int SYS, class R>
struct Tile3F {
  static constexpr int TY = 8;
  static constexpr int threads = kTX3 * TY;
  static constexpr int UH = TY + 6, NH = TY + 4;  // U tile + 3, nu tile + 2
  static constexpr int halo = 2 * TY + 2 * kTX3;  // halo columns and rows that stream into the tile
  // resident blocks per SM the registers are budgeted for (two blocks of 8
  // rows fit in shared memory only without the reactive field)
  static constexpr int min_blocks = (TY == 8 && sizeof(R) == 4 && SYS != SYS_REACT) ? 2 : 1;
};

// The own columns' f^n through one TMA box per plane in FP32.  FP64 (bound by
// the FP64 pipe) loads it where it is used: the box would not fit beside the
// U ring at every system.
template <class R>
constexpr bool k3f_f_tma() {
  return sizeof(R) == 4;
}

template <int SYS, class R>
struct Smem3F {
  static constexpr int M = Fields3<SYS>::M, TY = Tile3F<SYS, R>::TY;
  static constexpr int UH = Tile3F<SYS, R>::UH, NH = Tile3F<SYS, R>::NH;
  static constexpr size_t a128(size_t b) { return (b + 127) / 128 * 128; }
  static constexpr uint32_t u_box = (uint32_t)(M * UH * kUW3 * sizeof(R));  // bytes of one U box
  static constexpr uint32_t f_box = (uint32_t)(7 * M * TY * kTX3 * sizeof(R));
  static constexpr size_t u_slot = a128(u_box);  // TMA destinations start on 128 bytes
  static constexpr size_t f_off = kURing3 * u_slot;
  static constexpr size_t nu_off = f_off + (k3f_f_tma<R>() ? a128(f_box) : 0);
  static constexpr size_t py_off = nu_off + (size_t)NH * kNW3 * sizeof(R);
  static constexpr size_t py_bytes = (size_t)M * (TY + 1) * kTX3 * sizeof(R);
  static constexpr size_t my_off = py_off + py_bytes;
  static constexpr size_t hx_off = my_off + py_bytes;
  static constexpr size_t hf_off = hx_off + (size_t)2 * M * TY * sizeof(R);
  static constexpr size_t bar_off = (hf_off + (size_t)Tile3F<SYS, R>::halo * M * sizeof(R) + 7) / 8 * 8;
  // plus 128 bytes of slack: the kernel starts its layout on the first
  // 128-byte boundary of its dynamic shared memory
  static constexpr size_t total = bar_off + (kURing3 + 1) * sizeof(unsigned long long) + 128;
};

__device__ __forceinline__ void tma_load_box3(const CUtensorMap* tm, uint32_t dst, uint32_t bar, int x, int y, int z,
                                              uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_box4(const CUtensorMap* tm, uint32_t dst, uint32_t bar, int x, int y, int z,
                                              int w, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

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

// tu0/tu1: U copies 0/1 as {ex, ey, ez, m} (rows of G.px elements), boxes
// {40, TY + 6, 1, m}; tf0/tf1: distribution buffers 0/1 as {pitch, ny * nz,
// 7 m}, boxes {32, TY, 7 m}
template <int SYS, class R>
__global__ void __launch_bounds__(Tile3F<SYS, R>::threads, Tile3F<SYS, R>::min_blocks)
    k3_fused(const __grid_constant__ CUtensorMap tu0, const __grid_constant__ CUtensorMap tu1,
             const __grid_constant__ CUtensorMap tf0, const __grid_constant__ CUtensorMap tf1, DevParams P,
             R* const* buf, Ctl* ctl, int slot, ExtGeom3 G, R* Ue2, double* partials, int zc) {
  constexpr int M = Fields3<SYS>::M, Q = 7;
  constexpr bool SRC = SYS == SYS_REACT;
  constexpr bool FBOX = k3f_f_tma<R>();
  using L = Smem3F<SYS, R>;
  constexpr int TY = Tile3F<SYS, R>::TY, NT = Tile3F<SYS, R>::threads;
  constexpr int UH = Tile3F<SYS, R>::UH, NH = Tile3F<SYS, R>::NH;
  constexpr int NHALO = Tile3F<SYS, R>::halo;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* const smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  const R* fs = (const R*)(smem_raw + L::f_off);  // [7 m][TY][kTX3]
  R* nus = (R*)(smem_raw + L::nu_off);            // [NH][kNW3]: nu summed over planes q-3..q-1
  R* pys = (R*)(smem_raw + L::py_off);            // [M][TY + 1][kTX3]
  R* mys = (R*)(smem_raw + L::my_off);            // [M][TY + 1][kTX3]
  R* hxs = (R*)(smem_raw + L::hx_off);            // [2][M][TY]
  R* hfs = (R*)(smem_raw + L::hf_off);            // [NHALO][M]
  unsigned long long* bars = (unsigned long long*)(smem_raw + L::bar_off);  // U slots 0..3, f box 4
  __shared__ StepCoef3 s_cf;
  __shared__ R s_k[10];  // a0, 1/(2 lambda), dt/2, alpha_0..2, a_1..3, a0lo
  __shared__ int s_abort;
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
    const RestCoef<R> rc = rest_coef<R>(c.a0, &s_k[3], 3, s_k[1]);
    s_k[0] = rc.hi;
    s_k[9] = rc.lo;
    for (int i = 0; i < kURing3 + 1; i++) mbar_init(smem_u32(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
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
  R* Uo_ext = ue_copy<M>(Ue2, G, par ^ 1);  // U^{n+1} of the interior, for the next step
  const CUtensorMap* tu = par ? &tu1 : &tu0;
  const CUtensorMap* tf = par ? &tf1 : &tf0;
  const long long n = G.size();
  const long long nf = 7ll * M * P.plane;
  unsigned int* const stc = &ctl->status;
  const Phys<R> K = make_phys<R>(P);
  const R a0 = s_k[0], a0lo = s_k[9], inv2l = s_k[1], hdt = s_k[2];
  const R al[3] = {s_k[3], s_k[4], s_k[5]};
  const R aj[3] = {s_k[6], s_k[7], s_k[8]};
  const bool fixed_omega = P.omega_mode == 1;
  R om_fixed;
  if constexpr (sizeof(R) == 4)
    om_fixed = P.pf.omega_fixed;
  else
    om_fixed = P.omega_fixed;

  const int x0 = blockIdx.x * kTX3, y0 = blockIdx.y * TY;
  const int zb = blockIdx.z * zc, ze = min(zb + zc, P.nz3);
  const int x = x0 + tx, y = y0 + ty;
  const bool own_valid = x < P.nx && y < P.ny3;
  const int mx = map_index(x, P.nx, P.bc[0], P.bc[1]), my = map_index(y, P.ny3, P.bc[2], P.bc[3]);
  const int q0 = zb - 3, q1 = ze + 2;

  // U(p) on the tile + 3 (ext coordinates x0.., y0.., p + GH) into ring slot
  // (p - q0) % 4; points past the extension arrive as zeros and are never
  // used for an output
  auto uslot = [&](int p) -> const R* { return (const R*)(smem_raw + (size_t)((p - q0) % kURing3) * L::u_slot); };
  auto issue_u = [&](int p) {
    const int s = (p - q0) % kURing3;
    tma_load_box4(tu, smem_u32(smem_raw + (size_t)s * L::u_slot), smem_u32(&bars[s]), x0, y0, p + GH, 0, L::u_box);
  };
  // f^n of the own columns of plane pp (mapped to mk): rows mk * ny + y0..
  auto issue_f = [&](int pp) {
    const int mk = map_index(pp, P.nz3, P.bc_z[0], P.bc_z[1]);
    tma_load_box3(tf, smem_u32(smem_raw + L::f_off), smem_u32(&bars[kURing3]), XPAD + x0, mk * P.ny3 + y0, 0,
                  L::f_box);
  };

  // this thread's halo node (t < NHALO): the one direction qq (along dir) it
  // streams into the tile
  int hx = 0, hy = 0, hq = 0, hdir = 0;
  if (t < TY) { hx = -1; hy = t; hq = 1; hdir = 0; }
  else if (t < 2 * TY) { hx = kTX3; hy = t - TY; hq = 4; hdir = 0; }
  else if (t < 2 * TY + kTX3) { hx = t - 2 * TY; hy = -1; hq = 2; hdir = 1; }
  else if (t < NHALO) { hx = t - 2 * TY - kTX3; hy = TY; hq = 5; hdir = 1; }
  const int hmx = map_index(x0 + hx, P.nx, P.bc[0], P.bc[1]), hmy = map_index(y0 + hy, P.ny3, P.bc[2], P.bc[3]);

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
  // nu of this thread's phase-1 positions (t, t + NT, ...) on the two planes
  // before the one being computed
  constexpr int NUI = (NH * kNW3 + NT - 1) / NT;
  R nu3[NUI], nu2[NUI];
#pragma unroll
  for (int i = 0; i < NUI; i++) nu3[i] = nu2[i] = R(0);

  // load bookkeeping of thread 0, the issuing thread: it issues a load only
  // while every wait it made has succeeded, and before exiting waits for every
  // load it issued and has not seen land (a CTA whose wait gave up leaves no
  // copy in flight)
  int u_issued = q0 - 1, u_seen = q0 - 1;
  int f_issued = 0, f_seen = 0;
  unsigned f_waits = 0;
  bool ok0 = true;
  if (t == 0) {
    issue_u(q0);
    u_issued = q0;
    if (FBOX && zb + 1 <= q1) {
      issue_f(zb - 1);
      f_issued = 1;
    }
  }

#pragma unroll 1
  for (int q = q0; q <= q1; q++) {
    const bool got = mbar_wait_bounded(smem_u32(&bars[(q - q0) % kURing3]), (unsigned)((q - q0) / kURing3) & 1u);
    if (!got) s_abort = 1;
    if (t == 0) {
      if (got) u_seen = q;
      ok0 = ok0 && got;
      if (ok0 && q < q1) {  // slot (q + 1 - q0) % 4 last held U(q - 3): read for the last time in plane q - 1
        issue_u(q + 1);
        u_issued = q + 1;
      }
    }
    const bool posts = q >= zb + 1;
    const int pp = q - 2;  // plane of this iteration's posts
    const int mk = map_index(pp, P.nz3, P.bc_z[0], P.bc_z[1]);
    if (posts && t < NHALO) {  // the halo node's f^n of its direction, for phase 3
      const long long off = cell3(P, hmx, hmy, mk);
#pragma unroll
      for (int c = 0; c < M; c++)
        cp_async_elem(hfs + t * M + c, f + chk((long long)(hq * M + c) * P.plane + off, nf, stc));
      cp_async_commit();
    }
    // no block barrier here: each thread waited for U(q) itself, and every
    // buffer phase 1 writes was last read before the previous plane's barriers
    // 1: nu(q - 1) on the tile + 2
    if (q >= zb - 1) {
      const R* Um1 = uslot(q - 2);
      const R* U00 = uslot(q - 1);
      const R* Up1 = uslot(q);
#pragma unroll
      for (int i = 0; i < NUI; i++) {
        const int it = t + i * NT;
        if (it >= NH * kNW3) break;
        const int iy = it / kNW3, ix = it % kNW3;
        const int o = (iy + 1) * kUW3 + (ix + 1);  // position in the U tile
        constexpr int CS = UH * kUW3;
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
        nus[it] = (nu3[i] + nu2[i]) + sum;  // planes q-3, q-2, q-1 (garbage before q = zb + 1, never read)
        nu3[i] = nu2[i];
        nu2[i] = sum;
      }
    }
    __syncthreads();
    if (s_abort) break;  // a wait gave up (set before this barrier, read by all after it)
    // 2: omega(q - 2) at a position (jy, jx) of the tile + 1, by the thread
    // whose post needs it (the z-summed nu in the order (bj, bi)): no shared
    // omega plane and no barrier of its own
    auto omega_at = [&](int jy, int jx) -> R {
      if (fixed_omega) return om_fixed;
      R s = R(0);
#pragma unroll
      for (int bj = 0; bj < 3; bj++)
#pragma unroll
        for (int bi = 0; bi < 3; bi++) s += nus[(jy + bj) * kNW3 + jx + bi];
      return R(1) + fdiv(R(1), R(1) + s);
    };
    if (posts) {
      // 3: posts of plane pp = q - 2
      const R* Ut = uslot(pp);
      constexpr int CS = UH * kUW3;
      // own column: all seven directions
      R pown[Q][M];
      {
        R U[M], fq[Q][M], S[M], F[3][M];
        const int o = (ty + 3) * kUW3 + (tx + 3);
#pragma unroll
        for (int c = 0; c < M; c++) U[c] = Ut[c * CS + o];
        const R w = omega_at(ty + 1, tx + 1);
        if constexpr (FBOX) {
          const bool fgot = mbar_wait_bounded(smem_u32(&bars[kURing3]), f_waits & 1u);
          f_waits++;
          if (!fgot) s_abort = 1;
          if (t == 0) {
            if (fgot) f_seen++;
            ok0 = ok0 && fgot;
          }
          if (own_valid) {
#pragma unroll
            for (int k = 0; k < Q; k++)
#pragma unroll
              for (int c = 0; c < M; c++) fq[k][c] = fs[(k * M + c) * (TY * kTX3) + ty * kTX3 + tx];
          } else {  // a lane past the lattice's edge (ragged tile): its ghost node is the mapped node
            const long long off = cell3(P, mx, my, mk);
#pragma unroll
            for (int k = 0; k < Q; k++)
#pragma unroll
              for (int c = 0; c < M; c++) fq[k][c] = f[chk((long long)(k * M + c) * P.plane + off, nf, stc)];
          }
        } else {
          const long long off = cell3(P, mx, my, mk);
#pragma unroll
          for (int k = 0; k < Q; k++)
#pragma unroll
            for (int c = 0; c < M; c++) fq[k][c] = f[chk((long long)(k * M + c) * P.plane + off, nf, stc)];
        }
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
          R v = fq[0][c] - w * (fq[0][c] - rest_eq(a0, a0lo, U[c]));
          if constexpr (SRC) {
            if (src_field<SYS, 3>(c)) v += hdt * a0 * S[c];
          }
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
              if (src_field<SYS, 3>(c)) {
                vp += hdt * aj[d] * S[c];
                vm += hdt * aj[d] * S[c];
              }
            }
            pown[1 + d][c] = vp;
            pown[4 + d][c] = vm;
          }
      }
#pragma unroll
      for (int c = 0; c < M; c++) {
        pys[(c * (TY + 1) + ty + 1) * kTX3 + tx] = pown[2][c];
        mys[(c * (TY + 1) + ty) * kTX3 + tx] = pown[5][c];
      }
      // halo: the one direction each halo column / row streams into the tile
      if (t < NHALO) {
        cp_async_wait_all();  // this thread's own copies of its halo f^n
        const int o = (hy + 3) * kUW3 + (hx + 3);
        R U[M], fq[M], S[M], F[M];
#pragma unroll
        for (int c = 0; c < M; c++) {
          U[c] = Ut[c * CS + o];
          fq[c] = hfs[t * M + c];
        }
        const R w = omega_at(hy + 1, hx + 1);
        const Prim3<R> pw = prim3<SYS, R>(K, U);
        if constexpr (SRC)
          source3<SYS, R>(K, U, S);
        else
#pragma unroll
          for (int c = 0; c < M; c++) S[c] = R(0);
        flux3<SYS, R>(K, P, U, pw, hdir, F);
        const R alh = hdir == 0 ? al[0] : al[1], ajh = hdir == 0 ? aj[0] : aj[1];  // selected, not indexed
        R* dst = hq == 1 ? hxs + hy : (hq == 4 ? hxs + M * TY + hy : (hq == 2 ? pys + hx : mys + TY * kTX3 + hx));
        const int cstride = (hq == 1 || hq == 4) ? TY : (TY + 1) * kTX3;
#pragma unroll
        for (int c = 0; c < M; c++) {
          const R feq = hq <= 3 ? (alh * U[c] + F[c]) * inv2l : (alh * U[c] - F[c]) * inv2l;
          R v = fq[c] - w * (fq[c] - feq);
          if constexpr (SRC) {
            if (src_field<SYS, 3>(c)) v += hdt * ajh * S[c];
          }
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
        // the second half-source dt/2 a_k S(U^{n+1}): Eq. (2.8) makes
        // dt/2 S_5(U^{n+1}) = (rho Y)^{n+1} - (rho Y)bar, so S is not evaluated again
        R hs = R(0);
        if constexpr (SRC) {
          if (K.react && Ubar[5] != R(0)) {
            R z;
            st |= react_implicit3<R>(K, Ubar, cf.dt, hdt, &z);
            hs = z - Ubar[5];
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
            if constexpr (SRC) {
              if (src_field<SYS, 3>(c)) v += akq * hs;
            }
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
      __syncthreads();  // the sideways posts of plane q - 2 are in shared memory; the f box is read
      if (FBOX && t == 0 && ok0 && q + 1 <= q1) {  // the own f^n of plane q - 1, for the next plane's posts
        issue_f(q - 1);
        f_issued++;
      }
      // gather them for plane q - 2 (streamed one plane later)
#pragma unroll
      for (int c = 0; c < M; c++) {
        const R left = __shfl_up_sync(0xffffffffu, pown[1][c], 1);
        const R right = __shfl_down_sync(0xffffffffu, pown[4][c], 1);
        kxp[c] = tx == 0 ? hxs[c * TY + ty] : left;
        kxm[c] = tx == 31 ? hxs[(M + c) * TY + ty] : right;
        kyp[c] = pys[(c * (TY + 1) + ty) * kTX3 + tx];
        kym[c] = mys[(c * (TY + 1) + ty + 1) * kTX3 + tx];
        kp0[c] = pown[0][c];
        pz2[c] = pz1[c];
        pz1[c] = pown[3][c];
      }
    }
  }
  cp_async_wait_all();
  if (t == 0) {  // loads issued and not seen landing: only after a wait gave up
    bool drained = true;
    for (int p = u_seen + 1; p <= u_issued; p++)
      drained = mbar_wait_bounded(smem_u32(&bars[(p - q0) % kURing3]), (unsigned)((p - q0) / kURing3) & 1u) && drained;
    for (int i = f_seen; i < f_issued; i++) drained = mbar_wait_bounded(smem_u32(&bars[kURing3]), (unsigned)i & 1u) && drained;
    if (!drained) st |= ST_TIMEOUT;
  }
  if (s_abort) st |= ST_TIMEOUT;
  // side outputs per warp (partial slot bid * 8 + warp): no block barrier
  warp_side_outputs3<M, R>(sp0, sp1, sp2, acc, ctl, (slot + 1) % 3,
                           partials + (bid * (NT / 32) + ty) * M, st);
  if (bid == 0 && t == 0) advance_ctl3(ctl, slot, cf);
}

// launch shape of the fused 3D step: tiles of 32 x ty columns, chunks of zc planes
inline dim3 grid3_fused(int nx, int ny, int nz, int ty, int zc) {
  return dim3((unsigned)((nx + kTX3 - 1) / kTX3), (unsigned)((ny + ty - 1) / ty), (unsigned)((nz + zc - 1) / zc));
}

// TMA descriptors of the fused 3D step: both U copies of the ghost-extended
// grid and both distribution buffers (layouts as described at k3_fused)
template <int SYS, class R>
inline int k3f_encode_maps(FusedPlan& fp, const DevParams& P, const ExtGeom3& G, void* Ue2, void* const* fbuf) {
  constexpr int M = Fields3<SYS>::M, TY = Tile3F<SYS, R>::TY;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return -1;
  const CUtensorMapDataType dt = sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t s = sizeof(R);
  for (int b = 0; b < 2; b++) {
    cuuint64_t udims[4] = {(cuuint64_t)G.ex, (cuuint64_t)G.ey, (cuuint64_t)G.ez, (cuuint64_t)M};
    cuuint64_t ustr[3] = {(cuuint64_t)G.px * s, (cuuint64_t)G.px * G.ey * s, (cuuint64_t)G.size() * s};
    cuuint32_t ubox[4] = {(cuuint32_t)kUW3, (cuuint32_t)Tile3F<SYS, R>::UH, 1u, (cuuint32_t)M};
    cuuint32_t e4[4] = {1u, 1u, 1u, 1u};
    CUresult r = enc(&fp.tu3[b], dt, 4, (R*)Ue2 + (size_t)b * M * G.size(), udims, ustr, ubox, e4,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -1;
    cuuint64_t fdims[3] = {(cuuint64_t)P.pitch, (cuuint64_t)P.ny, (cuuint64_t)(7 * M)};
    cuuint64_t fstr[2] = {(cuuint64_t)P.pitch * s, (cuuint64_t)P.plane * s};
    cuuint32_t fbox[3] = {(cuuint32_t)kTX3, (cuuint32_t)TY, (cuuint32_t)(7 * M)};
    cuuint32_t e3[3] = {1u, 1u, 1u};
    r = enc(&fp.tf3[b], dt, 3, fbuf[b], fdims, fstr, fbox, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -1;
  }
  return 0;
}

}  // namespace lbmh
