// Fused single-pass collide-and-stream kernels.
//
// Every distribution is read from HBM once and written once per step; all
// intermediate quantities (U on the 3-node halo, nu, omega, post-collision
// values) live in registers or shared memory.
//
// 2D (D2Q5): a CTA of 128 threads owns a strip of 120 output columns and
// marches down the rows of a contiguous chunk of (strip, row) work.  Lane t
// holds global column x0 - 4 + t, so the 3-column halo on each side (plus one
// spare column for 16-byte alignment) is covered without a second pass.  One
// TMA load (cp.async.bulk.tensor, box {128 columns, 1 row, Q*m planes}) brings
// a whole row of f^n into a shared-memory ring of 3 + P rows, P rows ahead of
// use; the rows above and below come from the ring, so each row is fetched
// once.  Per loaded row r:
//   B  U(r) = sum_k f_k                          (Eq. 2.3)
//   C  nu(r-1) from U(r-2), U(r-1) +- 1 col, U(r) (Eq. 2.13, 2.14)
//   D  omega(r-2) from the 3x3 box of nu (2.15, 2.16); post(r-2) (2.2, 2.20)
//   E  row r-3: pull streaming, implicit moment (2.8), second half-source,
//      store f^{n+1}; side outputs (speed bound for the next step, FP64 sums)
// 1D (D1Q3): one CTA per 120-node chunk, everything in shared memory.
#pragma once
#include <cuda.h>

#include "physics.cuh"
#include "unfused.cuh"

namespace lbmh {

constexpr int FT = 128;          // threads per CTA = columns per loaded row
constexpr int FW = FT - 8;       // output columns per strip
constexpr int FPREF = 2;         // rows in flight ahead of use

struct FusedPlan {
  int blocks;      // grid size
  int strips;      // ceil(nx / FW) (2D)
  int smem;        // dynamic shared memory bytes
  CUtensorMap tm[2];
};

template <int SYS, int D, class R>
constexpr bool fused_available() { return true; }

template <int M, class R, int PREF>
struct Smem2D {
  static constexpr int QM = 5 * M, S = 3 + PREF;
  static constexpr size_t f_bytes = (size_t)S * QM * FT * sizeof(R);
  static constexpr size_t u_bytes = (size_t)2 * M * FT * sizeof(R);
  static constexpr size_t c_bytes = (size_t)FT * sizeof(R);
  static constexpr size_t p_bytes = (size_t)2 * 2 * M * FT * sizeof(R);
  static constexpr size_t bar_off = f_bytes + u_bytes + c_bytes + p_bytes;
  static constexpr size_t total = bar_off + S * sizeof(unsigned long long);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: gives up after ~2^22 polls (each try_wait may itself sleep)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_row(const CUtensorMap* tm, uint32_t dst, uint32_t bar, int x, int y,
                                             uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(tm), "r"(x), "r"(y), "r"(0), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

template <int SYS, class R, int PREF>
__global__ void __launch_bounds__(FT) k_fused2d(const __grid_constant__ CUtensorMap tm0,
                                                const __grid_constant__ CUtensorMap tm1, DevParams P,
                                                R* const* buf, Ctl* ctl, int slot, double* partials, int strips) {
  constexpr int M = Fields<SYS, 2>::M, Q = 5, QM = Q * M;
  using L = Smem2D<M, R, PREF>;
  constexpr int S = L::S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* fring = (R*)smem_raw;
  R* Usm = (R*)(smem_raw + L::f_bytes);
  R* colsm = (R*)(smem_raw + L::f_bytes + L::u_bytes);
  R* p13 = (R*)(smem_raw + L::f_bytes + L::u_bytes + L::c_bytes);
  unsigned long long* bars = (unsigned long long*)(smem_raw + L::bar_off);
  __shared__ int s_abort;

  const int t = threadIdx.x;
  const StepCoef cf = step_coef<2>(P, ctl, slot);
  if (!cf.active) {
    if (blockIdx.x == 0 && t == 0) advance_ctl<2>(ctl, slot, cf);
    return;
  }
  const int par = ctl->parity[slot];
  const CUtensorMap* tm = par ? &tm1 : &tm0;
  const R* fin = buf[par];
  R* fout = buf[par ^ 1];

  if (t == 0) {
    for (int i = 0; i < S; i++) mbar_init(smem_u32(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();

  const R a0 = R(cf.a0), inv2l = R(1.0 / (2.0 * cf.lam)), hdt = R(0.5 * cf.dt);
  const R al0 = R(cf.alpha[0]), al1 = R(cf.alpha[1]);
  const R akk[5] = {R(cf.a0), R(cf.aj[0]), R(cf.aj[1]), R(cf.aj[0]), R(cf.aj[1])};
  const R dxr = R(P.dx);
  const bool fixed_omega = P.omega_mode == 1;
  const R om_fixed = R(P.omega_fixed);
  const uint32_t row_bytes = (uint32_t)(QM * FT * sizeof(R));

  double sp0 = 0.0, sp1 = 0.0, usum[M];
#pragma unroll
  for (int c = 0; c < M; c++) usum[c] = 0.0;
  unsigned st = 0u;

  const long long total = (long long)strips * P.ny;
  const long long wb = total * blockIdx.x / gridDim.x, we = total * (blockIdx.x + 1) / gridDim.x;
  unsigned seq = 0;
  bool aborted = false;

  for (long long w = wb; w < we && !aborted;) {
    const int strip = (int)(w / P.ny);
    const int yb = (int)(w % P.ny);
    const int ye = (int)min((long long)P.ny, (long long)yb + (we - w));
    w += ye - yb;
    const int x0 = strip * FW;
    const int gx = x0 - 4 + t;
    const bool col_in = gx >= 0 && gx < P.nx;
    const int mx = map_index(gx, P.nx, P.bc[0], P.bc[1]);
    const bool out_col = t >= 4 && t < FT - 4 && gx < P.nx;
    const double xpos = P.x0 + (mx + 0.5) * P.dx;
    const int r0 = yb - 3, r1 = ye + 2;
    const unsigned seq0 = seq;
    seq += (unsigned)(r1 - r0 + 1);

    unsigned issued_end = seq0;  // one past the last row copy issued (thread 0)
    if (t == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int i = 0; i < PREF && r0 + i <= r1; i++) {
        unsigned s = seq0 + i;
        int my = map_index(r0 + i, P.ny, P.bc[2], P.bc[3]);
        tma_load_row(tm, smem_u32(fring + (size_t)(s % S) * QM * FT), smem_u32(&bars[s % S]), x0 - 4, my, row_bytes);
        issued_end = s + 1;
      }
    }
    unsigned cur = seq0;

    R U1[M], U2[M], p0[M], p2a[M], p2b[M];
#pragma unroll
    for (int c = 0; c < M; c++) U1[c] = U2[c] = p0[c] = p2a[c] = p2b[c] = R(0);
    R nu1 = R(0), nu2 = R(0), nu3 = R(0);

    for (int r = r0; r <= r1; r++) {
      const unsigned sidx = seq0 + (unsigned)(r - r0);
      cur = sidx;
      if (t == 0 && r + PREF <= r1) {
        unsigned s = sidx + PREF;
        int my = map_index(r + PREF, P.ny, P.bc[2], P.bc[3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tma_load_row(tm, smem_u32(fring + (size_t)(s % S) * QM * FT), smem_u32(&bars[s % S]), x0 - 4, my, row_bytes);
        issued_end = s + 1;
      }
      if (!mbar_wait_bounded(smem_u32(&bars[sidx % S]), (sidx / S) & 1u)) s_abort = 1;
      R* frow = fring + (size_t)(sidx % S) * QM * FT;
      const int myr = map_index(r, P.ny, P.bc[2], P.bc[3]);
      if (!col_in) {  // ghost column: copy of the wrapped / clamped node
        const R* src = fin + (long long)myr * P.pitch + mx;
#pragma unroll
        for (int q = 0; q < QM; q++) frow[q * FT + t] = src[(long long)q * P.plane];
      }
      // B: moments of row r
      R Ur[M];
#pragma unroll
      for (int c = 0; c < M; c++) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < Q; k++) s += frow[(k * M + c) * FT + t];
        Ur[c] = s;
        Usm[((r & 1) * M + c) * FT + t] = s;
      }
      // C: indicator of row r-1
      R nun = R(0);
      if (t >= 1 && t < FT - 1) {
        const R* Uprev = Usm + ((r - 1) & 1) * M * FT;
        R dm[M], dp[M];
        Prim<R> w1 = primitives<SYS, 2, R>(P, U1);
#pragma unroll
        for (int c = 0; c < M; c++) {
          dm[c] = U1[c] - Uprev[c * FT + t - 1];
          dp[c] = Uprev[c * FT + t + 1] - U1[c];
        }
        nun = theta_sum<SYS, 2, R>(P, w1, 0, dm, dp, dxr);
#pragma unroll
        for (int c = 0; c < M; c++) {
          dm[c] = U1[c] - U2[c];
          dp[c] = Ur[c] - U1[c];
        }
        nun += theta_sum<SYS, 2, R>(P, w1, 1, dm, dp, dxr);
      }
      nu3 = nu2;
      nu2 = nu1;
      nu1 = nun;
      colsm[t] = nu1 + nu2 + nu3;
      __syncthreads();
      if (s_abort) {
        aborted = true;
        break;
      }
      // D: omega and post-collision values of row r-2
      R om = om_fixed;
      if (!fixed_omega && t >= 1 && t < FT - 1) om = R(1) + fdiv(R(1), R(1) + (colsm[t - 1] + colsm[t] + colsm[t + 1]));
      const R* f2 = fring + (size_t)(((sidx % S) + S - 2) % S) * QM * FT;
      R post[Q][M];
      {
        Prim<R> w2 = primitives<SYS, 2, R>(P, U2);
        R Fx[M], Fy[M], Sr[M];
        flux<SYS, 2, R>(P, U2, w2, 0, Fx);
        flux<SYS, 2, R>(P, U2, w2, 1, Fy);
        const int my2 = map_index(r - 2, P.ny, P.bc[2], P.bc[3]);
        source<SYS, 2, R>(P, U2, xpos, P.y0 + (my2 + 0.5) * P.dx, Sr);
#pragma unroll
        for (int c = 0; c < M; c++) {
          R feq[Q];
          feq[0] = a0 * U2[c];
          feq[1] = (al0 * U2[c] + Fx[c]) * inv2l;
          feq[2] = (al1 * U2[c] + Fy[c]) * inv2l;
          feq[3] = (al0 * U2[c] - Fx[c]) * inv2l;
          feq[4] = (al1 * U2[c] - Fy[c]) * inv2l;
#pragma unroll
          for (int k = 0; k < Q; k++) {
            R fk = f2[(k * M + c) * FT + t];
            post[k][c] = fk - om * (fk - feq[k]) + hdt * akk[k] * Sr[c];
          }
        }
      }
      R* p13w = p13 + (((r - 2) & 1) * 2) * M * FT;
#pragma unroll
      for (int c = 0; c < M; c++) {
        p13w[c * FT + t] = post[1][c];
        p13w[(M + c) * FT + t] = post[3][c];
      }
      // E: row r-3
      const int y = r - 3;
      if (out_col && y >= yb && y < ye) {
        const R* p13r = p13 + (((r - 3) & 1) * 2) * M * FT;
        R Fk[Q][M], Ubar[M], Un[M], Sn[M];
#pragma unroll
        for (int c = 0; c < M; c++) {
          Fk[0][c] = p0[c];
          Fk[1][c] = p13r[c * FT + t - 1];
          Fk[2][c] = p2a[c];
          Fk[3][c] = p13r[(M + c) * FT + t + 1];
          Fk[4][c] = post[4][c];
          R s = R(0);
#pragma unroll
          for (int k = 0; k < Q; k++) s += Fk[k][c];
          Ubar[c] = s;
        }
        const double ypos = P.y0 + (y + 0.5) * P.dx, xo = P.x0 + (gx + 0.5) * P.dx;
        st |= implicit_moment<SYS, 2, R>(P, Ubar, xo, ypos, cf.dt, Un);
        source<SYS, 2, R>(P, Un, xo, ypos, Sn);
        R Us[M];
        const long long off = (long long)y * P.pitch + gx;
#pragma unroll
        for (int c = 0; c < M; c++) Us[c] = R(0);
#pragma unroll
        for (int k = 0; k < Q; k++)
#pragma unroll
          for (int c = 0; c < M; c++) {
            R v = Fk[k][c] + hdt * akk[k] * Sn[c];
            fout[(long long)(k * M + c) * P.plane + off] = v;
            Us[c] += v;
          }
        Prim<R> wn = primitives<SYS, 2, R>(P, Us);
        sp0 = fmax(sp0, (double)max_speed<SYS, 2, R>(P, wn, 0));
        sp1 = fmax(sp1, (double)max_speed<SYS, 2, R>(P, wn, 1));
#pragma unroll
        for (int c = 0; c < M; c++) usum[c] += (double)Us[c];
        st |= state_status<SYS, 2, R>(P, Us);
      }
#pragma unroll
      for (int c = 0; c < M; c++) {
        p0[c] = post[0][c];
        p2a[c] = p2b[c];
        p2b[c] = post[2][c];
        U2[c] = U1[c];
        U1[c] = Ur[c];
      }
      __syncthreads();
    }
    if (aborted) {
      // let every row copy this CTA issued land before the CTA exits
      if (t == 0)
        for (unsigned s = cur; s < issued_end; s++) mbar_wait_bounded(smem_u32(&bars[s % S]), (s / S) & 1u);
      st |= ST_TIMEOUT;
      __syncthreads();
    }
  }
  block_side_outputs<M>(sp0, sp1, usum, ctl, (slot + 1) % 3, partials, st);
  if (blockIdx.x == 0 && t == 0) advance_ctl<2>(ctl, slot, cf);
}

// 1D: one CTA per chunk of FW nodes; lane t holds node x0 - 4 + t
template <int SYS, class R>
__global__ void __launch_bounds__(FT) k_fused1d(DevParams P, R* const* buf, Ctl* ctl, int slot, double* partials) {
  constexpr int M = Fields<SYS, 1>::M, Q = 3;
  __shared__ R Us[M][FT];
  __shared__ R nus[FT];
  __shared__ R p1s[M][FT], p2s[M][FT];
  const int t = threadIdx.x;
  const StepCoef cf = step_coef<1>(P, ctl, slot);
  if (!cf.active) {
    if (blockIdx.x == 0 && t == 0) advance_ctl<1>(ctl, slot, cf);
    return;
  }
  const int par = ctl->parity[slot];
  const R* fin = buf[par];
  R* fout = buf[par ^ 1];
  const int gx = blockIdx.x * FW - 4 + t;
  const int mx = map_index(gx, P.nx, P.bc[0], P.bc[1]);
  R f[Q][M], U[M];
#pragma unroll
  for (int c = 0; c < M; c++) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < Q; k++) {
      f[k][c] = fin[(long long)(k * M + c) * P.plane + mx];
      s += f[k][c];
    }
    U[c] = s;
    Us[c][t] = s;
  }
  __syncthreads();
  Prim<R> w = primitives<SYS, 1, R>(P, U);
  R nu = R(0);
  if (t >= 1 && t < FT - 1) {
    R dm[M], dp[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      dm[c] = U[c] - Us[c][t - 1];
      dp[c] = Us[c][t + 1] - U[c];
    }
    nu = theta_sum<SYS, 1, R>(P, w, 0, dm, dp, R(P.dx));
  }
  nus[t] = nu;
  __syncthreads();
  R om = R(P.omega_fixed);
  if (P.omega_mode != 1 && t >= 1 && t < FT - 1) om = R(1) + fdiv(R(1), R(1) + (nus[t - 1] + nus[t] + nus[t + 1]));
  const R a0 = R(cf.a0), a1 = R(cf.aj[0]), inv2l = R(1.0 / (2.0 * cf.lam)), hdt = R(0.5 * cf.dt);
  const R al0 = R(cf.alpha[0]);
  R F[M], S[M], post0[M];
  flux<SYS, 1, R>(P, U, w, 0, F);
  source<SYS, 1, R>(P, U, P.x0 + (mx + 0.5) * P.dx, 0.0, S);
#pragma unroll
  for (int c = 0; c < M; c++) {
    R feq0 = a0 * U[c], feq1 = (al0 * U[c] + F[c]) * inv2l, feq2 = (al0 * U[c] - F[c]) * inv2l;
    post0[c] = f[0][c] - om * (f[0][c] - feq0) + hdt * a0 * S[c];
    p1s[c][t] = f[1][c] - om * (f[1][c] - feq1) + hdt * a1 * S[c];
    p2s[c][t] = f[2][c] - om * (f[2][c] - feq2) + hdt * a1 * S[c];
  }
  __syncthreads();
  double sp0 = 0.0, usum[M];
#pragma unroll
  for (int c = 0; c < M; c++) usum[c] = 0.0;
  unsigned st = 0u;
  if (t >= 4 && t < FT - 4 && gx < P.nx) {
    R Fk[Q][M], Ubar[M], Un[M], Sn[M], Uo[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      Fk[0][c] = post0[c];
      Fk[1][c] = p1s[c][t - 1];
      Fk[2][c] = p2s[c][t + 1];
      Ubar[c] = Fk[0][c] + Fk[1][c] + Fk[2][c];
    }
    const double xo = P.x0 + (gx + 0.5) * P.dx;
    st |= implicit_moment<SYS, 1, R>(P, Ubar, xo, 0.0, cf.dt, Un);
    source<SYS, 1, R>(P, Un, xo, 0.0, Sn);
    const R ak[3] = {a0, a1, a1};
#pragma unroll
    for (int c = 0; c < M; c++) Uo[c] = R(0);
#pragma unroll
    for (int k = 0; k < Q; k++)
#pragma unroll
      for (int c = 0; c < M; c++) {
        R v = Fk[k][c] + hdt * ak[k] * Sn[c];
        fout[(long long)(k * M + c) * P.plane + gx] = v;
        Uo[c] += v;
      }
    Prim<R> wn = primitives<SYS, 1, R>(P, Uo);
    sp0 = (double)max_speed<SYS, 1, R>(P, wn, 0);
#pragma unroll
    for (int c = 0; c < M; c++) usum[c] = (double)Uo[c];
    st |= state_status<SYS, 1, R>(P, Uo);
  }
  block_side_outputs<M>(sp0, 0.0, usum, ctl, (slot + 1) % 3, partials, st);
  if (blockIdx.x == 0 && t == 0) advance_ctl<1>(ctl, slot, cf);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

template <int SYS, class R>
inline size_t fused2d_smem() {
  return Smem2D<Fields<SYS, 2>::M, R, FPREF>::total;
}

template <int SYS, int D, class R>
inline int fused_setup(FusedPlan& fp, const DevParams& P, void* const* fbuf) {
  constexpr int M = Fields<SYS, D>::M, QM = Fields<SYS, D>::Q * M;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (D == 1) {
    fp.strips = 1;
    fp.smem = 0;
    fp.blocks = (P.nx + FW - 1) / FW;
    return 0;
  }
  fp.strips = (P.nx + FW - 1) / FW;
  size_t smem = fused2d_smem<SYS, R>();
  fp.smem = (int)smem;
  auto kern = k_fused2d<SYS, R, FPREF>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FT, smem) != cudaSuccess || per_sm < 1) return -1;
  long long total = (long long)fp.strips * P.ny;
  long long want = (long long)per_sm * sms;
  long long cap = (total + 7) / 8;  // at least ~8 rows per CTA
  fp.blocks = (int)(want < cap ? want : (cap < 1 ? 1 : cap));
  EncodeTiledFn enc = encode_fn();
  if (!enc) return -1;
  for (int b = 0; b < 2; b++) {
    cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)QM};
    cuuint64_t strides[2] = {(cuuint64_t)P.pitch * sizeof(R), (cuuint64_t)P.plane * sizeof(R)};
    cuuint32_t box[3] = {(cuuint32_t)FT, 1u, (cuuint32_t)QM};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(&fp.tm[b], sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                     fbuf[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -1;
  }
  return 0;
}

template <int SYS, int D, class R>
inline int fused_launch(const FusedPlan& fp, const DevParams& P, R* const* buf, Ctl* ctl, int slot, double* partials,
                        cudaStream_t stream) {
  if (D == 1) {
    k_fused1d<SYS, R><<<fp.blocks, FT, 0, stream>>>(P, buf, ctl, slot, partials);
  } else {
    k_fused2d<SYS, R, FPREF><<<fp.blocks, FT, fp.smem, stream>>>(fp.tm[0], fp.tm[1], P, buf, ctl, slot, partials,
                                                                 fp.strips);
  }
  return fp.blocks;
}

}  // namespace lbmh
