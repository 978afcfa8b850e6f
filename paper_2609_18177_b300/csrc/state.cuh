// Set-up and diagnostic kernels shared by the single-lattice handles, the
// allocation-free step and the batch engine: initial equilibrium (Eq. 2.20),
// speed bounds (Eq. 2.19), moments (Eq. 2.3), checkpoint copies and the ghost
// columns of padded rows.
#pragma once
#include "common.cuh"
#include "physics.cuh"
#include "unfused.cuh"

namespace lbmh {

constexpr int kBlock = 256;
inline unsigned blocks_for(long long n, int bs = kBlock) { return (unsigned)((n + bs - 1) / bs); }

// grid of the node loops that end in a maximum (speed bounds): grid-stride
// loops over at most 2048 blocks, so that the maximum costs one atomic per
// block instead of one per warp (contended atomics on one address serialise)
inline unsigned reduce_blocks_for(long long n) {
  unsigned b = blocks_for(n);
  return b < 2048u ? (b ? b : 1u) : 2048u;
}

// (s0, s1) := their maxima over the block (kBlock threads); thread 0 folds
// them into d0, d1
__device__ __forceinline__ void block_max2_to(double s0, double s1, unsigned long long* d0,
                                              unsigned long long* d1) {
  __shared__ double red[2][kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 = fmax(s0, __shfl_xor_sync(0xffffffffu, s0, o));
    s1 = fmax(s1, __shfl_xor_sync(0xffffffffu, s1, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
  }
  __syncthreads();
  if (w == 0) {
    s0 = lane < kBlock / 32 ? red[0][lane] : 0.0;
    s1 = lane < kBlock / 32 ? red[1][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 = fmax(s0, __shfl_xor_sync(0xffffffffu, s0, o));
      s1 = fmax(s1, __shfl_xor_sync(0xffffffffu, s1, o));
    }
    if (lane == 0) {
      atomic_max_nonneg(d0, s0);
      atomic_max_nonneg(d1, s1);
    }
  }
}


// speed bound (2.19) of a FP64 state U0 [m][ny][nx] -> ctl->ainit
template <int SYS, int D>
__global__ void __launch_bounds__(kBlock) k_init_speed(DevParams P, const double* U0, Ctl* ctl) {
  constexpr int M = Fields<SYS, D>::M;
  const long long nn = (long long)P.nx * P.ny;
  const Phys<double> K = make_phys<double>(P);
  double s0 = 0.0, s1 = 0.0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
       node += (long long)gridDim.x * blockDim.x) {
    double U[M];
#pragma unroll
    for (int c = 0; c < M; c++) U[c] = U0[c * nn + node];
    Prim<double> w = primitives<SYS, D, double>(K, U);
    s0 = fmax(s0, max_speed<SYS, D, double>(K, w, 0));
    if (D == 2) s1 = fmax(s1, max_speed<SYS, D, double>(K, w, 1));
  }
  block_max2_to(s0, s1, (unsigned long long*)&ctl->ainit[0], (unsigned long long*)&ctl->ainit[1]);
}

// f := f^eq(U0) with alpha^0, lambda^0 from ctl->ainit (Eq. 2.20); the speed
// bound of the stored state goes to slot 0 for the first step.
template <int SYS, int D, class R>
__global__ void __launch_bounds__(kBlock) k_init_eq(DevParams P, const double* U0, R* f, Ctl* ctl) {
  constexpr int M = Fields<SYS, D>::M, Q = Fields<SYS, D>::Q;
  const long long nn = (long long)P.nx * P.ny;
  double ab0 = ctl->ainit[0], ab1 = D == 2 ? ctl->ainit[1] : 0.0;
  double dt = P.cfl * P.dx / (D == 2 ? ab0 + ab1 : ab0);
  double lam = P.dx / dt;
  double al0 = ab0 + P.eps, al1 = D == 2 ? ab1 + P.eps : 0.0;
  const R inv2l = R(1.0 / (2.0 * lam));
  const R al[2] = {R(al0), R(al1)};
  const RestCoef<R> rc = rest_coef<R>(1.0 - (D == 2 ? al0 + al1 : al0) / lam, al, D, inv2l);
  const Phys<R> K = make_phys<R>(P);
  double s0 = 0.0, s1 = 0.0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
       node += (long long)gridDim.x * blockDim.x) {
    int j = (int)(node / P.nx), i = (int)(node % P.nx);
    R U[M], Us[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      U[c] = R(U0[c * nn + node]);
      Us[c] = R(0);
    }
    Prim<R> w = primitives<SYS, D, R>(K, U);
    long long off = cell(P, i, j);
#pragma unroll
    for (int k = 0; k < Q; k++) {
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
#pragma unroll
      for (int c = 0; c < M; c++) {
        f[chk((long long)(k * M + c) * P.plane + off, (long long)Q * M * P.plane, &ctl->status)] = feq[c];
        Us[c] += feq[c];
      }
    }
    Prim<R> ws = primitives<SYS, D, R>(K, Us);
    s0 = fmax(s0, (double)max_speed<SYS, D, R>(K, ws, 0));
    if (D == 2) s1 = fmax(s1, (double)max_speed<SYS, D, R>(K, ws, 1));
  }
  block_max2_to(s0, s1, &ctl->amax[0][0], &ctl->amax[0][1]);
}

// U = sum_k f_k into FP64 [m][ny][nx]
template <int M, int Q, class R>
__global__ void k_moments(DevParams P, R* const* buf, const Ctl* ctl, int slot, double* U) {
  unsigned int* st = (unsigned int*)&ctl->status;
  long long nn = (long long)P.nx * P.ny;
  long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= nn) return;
  const R* f = buf[ctl->parity[slot]];
  int j = (int)(node / P.nx), i = (int)(node % P.nx);
  long long off = cell(P, i, j);
#pragma unroll
  for (int c = 0; c < M; c++) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < Q; k++) s += f[chk((long long)(k * M + c) * P.plane + off, (long long)Q * M * P.plane, st)];
    U[c * nn + node] = (double)s;
  }
}

// f <-> FP64 [Q][m][ny][nx] (checkpointing)
template <class R>
__global__ void k_get_f(DevParams P, int QM, R* const* buf, const Ctl* ctl, int slot, double* out) {
  long long nn = (long long)P.nx * P.ny;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= nn * QM) return;
  const R* f = buf[ctl->parity[slot]];
  long long q = idx / nn, node = idx % nn;
  int j = (int)(node / P.nx), i = (int)(node % P.nx);
  out[idx] = (double)f[chk(q * P.plane + cell(P, i, j), (long long)QM * P.plane, (unsigned int*)&ctl->status)];
}

template <class R>
__global__ void k_set_f(DevParams P, int QM, R* f, const double* in, Ctl* ctl) {
  long long nn = (long long)P.nx * P.ny;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= nn * QM) return;
  long long q = idx / nn, node = idx % nn;
  int j = (int)(node / P.nx), i = (int)(node % P.nx);
  f[chk(q * P.plane + cell(P, i, j), (long long)QM * P.plane, &ctl->status)] = R(in[idx]);
}

// speed bound of the stored distributions -> slot 0 (after lbmh_set_f)
template <int SYS, int D, class R>
__global__ void __launch_bounds__(kBlock) k_speed_of_f(DevParams P, R* const* buf, Ctl* ctl) {
  constexpr int M = Fields<SYS, D>::M, Q = Fields<SYS, D>::Q;
  const long long nn = (long long)P.nx * P.ny;
  const Phys<R> K = make_phys<R>(P);
  const R* f = buf[ctl->parity[0]];
  double s0 = 0.0, s1 = 0.0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
       node += (long long)gridDim.x * blockDim.x) {
    int j = (int)(node / P.nx), i = (int)(node % P.nx);
    long long off = cell(P, i, j);
    R U[M];
#pragma unroll
    for (int c = 0; c < M; c++) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < Q; k++) s += f[chk((long long)(k * M + c) * P.plane + off, (long long)Q * M * P.plane, &ctl->status)];
      U[c] = s;
    }
    Prim<R> w = primitives<SYS, D, R>(K, U);
    s0 = fmax(s0, (double)max_speed<SYS, D, R>(K, w, 0));
    if (D == 2) s1 = fmax(s1, (double)max_speed<SYS, D, R>(K, w, 1));
  }
  block_max2_to(s0, s1, &ctl->amax[0][0], &ctl->amax[0][1]);
}

// ghost columns of every row := the wrapped / clamped node (after the
// distributions were written by something other than a fused 2D step)
template <class R>
__global__ void k_fill_pads(DevParams P, int QM, R* f, Ctl* ctl) {
  long long rows = (long long)P.ny * QM;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= rows * 2 * NGHOST) return;
  long long row = idx / (2 * NGHOST);
  int p = (int)(idx % (2 * NGHOST));
  int x = p < NGHOST ? p - NGHOST : P.nx + (p - NGHOST);
  int src = map_index(x, P.nx, P.bc[0], P.bc[1]);
  long long q = row / P.ny, j = row % P.ny;
  const long long base = q * P.plane + j * P.pitch + XPAD, nf = (long long)QM * P.plane;
  f[chk(base + x, nf, &ctl->status)] = f[chk(base + src, nf, &ctl->status)];
}

template <class R>
__global__ void k_extract_interior(DevParams P, ExtGeom G, const R* src_ext, double* out) {
  long long nn = (long long)P.nx * P.ny;
  long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int j = (int)(node / P.nx), i = (int)(node % P.nx);
  out[node] = (double)src_ext[G.idx(j + G.gy, i + GH)];
}

// Slabs of a lattice decomposed along y: copy the three padded rows
// [row, row + 3) of every distribution plane of the current state between the
// lattice and a contiguous block rows[QM][3][pitch] (to_rows: lattice -> block)
template <class R>
__global__ void k_halo_rows(DevParams P, int QM, R* const* buf, const Ctl* ctl, int slot, int row, R* rows,
                            int to_rows) {
  const long long per = 3ll * P.pitch;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= per * QM) return;
  R* f = buf[ctl->parity[slot]];
  const long long q = idx / per, r = idx % per;
  R* a = f + chk(q * P.plane + (long long)row * P.pitch + r, (long long)QM * P.plane, (unsigned int*)&ctl->status);
  if (to_rows)
    rows[idx] = *a;
  else
    *a = rows[idx];
}

}  // namespace lbmh
