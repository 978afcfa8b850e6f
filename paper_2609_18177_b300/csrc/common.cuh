// Shared device-side definitions of the lbmh CUDA library: problem constants,
// the per-handle step-control block and small helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmh {

enum { SYS_ADV = 0, SYS_EULER = 1, SYS_SWE = 2, SYS_REACT = 3 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2, BC_INFLOW = 3 };

// number of conserved fields m of each system in d dimensions
template <int SYS, int D>
struct Fields {
  static constexpr int M = SYS == SYS_ADV ? 1 : SYS == SYS_EULER ? D + 2 : SYS == SYS_SWE ? D + 1 : D + 3;
  static constexpr int Q = 2 * D + 1;  // DdQ(2d+1) lattice, Section 2.3
};

// Every row of a distribution plane starts with XPAD padding columns: node x
// sits at column offset x + XPAD, so interior rows start on a 32-byte sector
// in FP32.  The NGHOST columns on each side of the interior (x in [-4, 0) and
// [nx, nx+4)) are ghost nodes: the fused 2D kernel keeps them equal to the
// wrapped / clamped node after each step, so a row of any strip can be
// fetched with one in-bounds, aligned TMA box.
// The unfused kernels (unfused.cuh) address only columns [0, nx): every
// column they read or write is cell(P, i, j) with i = map_index(...) in
// [0, nx) for periodic, outflow and reflecting sides.  The allocation-free
// step relies on this to run them on unpadded [..][ny][nx] arrays, with
// pitch = nx and the base pointers shifted by -XPAD, which they never
// dereference.
constexpr int XPAD = 8;
constexpr int NGHOST = 4;

// Problem constants, passed by value to every kernel.
// FP32 copies of the physical constants, rounded once on the host: the FP32
// path reads them as they are (a conversion from the double fields on the
// device is an FP64-pipe instruction, and the compiler may repeat it per row
// instead of keeping the value in a register)
struct PhysConstF {
  float gamma, gm1, g, half_g, h_dry, cmin, q, adv0, adv1, dx;
  float bed_amp, bed_inv_w2, bed_m2_inv_w2, xb, yb, K, Ti;
  float omega_fixed;
  float adv2;  // advection speed along z (3D)
  float sponge_dx_over_w;
  float u_in[8];
};

struct DevParams {
  int nx, ny;        // ny = 1 in 1D
  int pitch;         // elements between rows of one distribution plane (>= nx + 2*XPAD)
  long long plane;   // elements between planes (ny * pitch)
  int bc[4];         // xlo, xhi, ylo, yhi
  double x0, y0, dx;
  double cfl, eps;
  double T;          // > 0: steps stop once t >= T
  long long max_steps;  // > 0: steps stop once this many were taken
  double adv[2];
  double gamma, g, h_dry;
  double bed_amp, bed_w2, bed_xc, bed_yc;
  double K, Ti, q;
  int has_bed;       // bed_amp != 0 (flags set on the host: a device test of
  int has_react;     // K != 0           a double would be an FP64 instruction)
  int omega_mode;    // 0 adaptive, 1 fixed
  double omega_fixed;
  double sponge_width;      // > 0: sponge over [x0, x0 + sponge_width] (omega blended toward 1)
  double sponge_dx_over_w;  // dx / sponge_width
  double u_in[8];           // conservative state of INFLOW ghost nodes
  int has_special_bc;       // some side is REFLECT or INFLOW
  // 3D (D3Q7): ny above counts rows = ny3 * nz3 (z outer), so the row-wise
  // kernels (moments, checkpoints) serve 3D lattices unchanged
  int ny3, nz3;
  int bc_z[2];
  double z0, adv_z;
  // Rows the 2D single-lattice step writes: [ywin0, ywin1) (the whole lattice,
  // 0..ny, except for a slab of a lattice decomposed along y, whose three rows
  // next to a neighbouring slab are halo rows: read, never written).  row0 is
  // the global index of local row 0 (0 except for slabs): node positions (the
  // bed source) use global rows, so a slab computes the bits of the whole
  // lattice.
  int ywin0, ywin1;
  int row0;
  // polls of each CTA's first row-load wait in the 2D row pipeline (1 << 22;
  // LBMH_TEST_FIRST_WAIT_POLLS at handle creation sets it, so that a test can
  // make a wait run out without disturbing the GPU)
  int first_wait_polls;
  PhysConstF pf;
};

// Step-control block in device memory.  Step n reads slot n % 3, folds the
// next step's speed bound into slot (n+1) % 3 and clears slot (n+2) % 3, so a
// sequence of launches needs no host round trip (the global maximum of
// Eq. (2.19) is a side output of the previous step).
struct Ctl {
  unsigned long long amax[3][2];  // bit patterns of non-negative doubles
  double t[3];
  long long nsteps[3];
  int parity[3];                  // distribution buffer holding the state
  int pad;
  double last_dt, last_lambda;    // of the most recent executed step
  double ainit[2];                // speed bound of the initial state U0
  unsigned int status;            // LBMH status bits, sticky
  unsigned int pad2;
  unsigned long long amax_z[3];  // 3D: speed bound along z per slot (bit pattern)
  double ainit_z;
};

// status bits: NONPHYSICAL (NaN/inf, rho <= 0 or p <= 0) fails lbmh_moments;
// NEGATIVE_DEPTH (shallow water h < -1e-12, which the scheme produces at
// wet-dry fronts: it is not positivity preserving) is reported only; BOUNDS
// (bounds-checked builds only) marks an index that left its array.
enum : unsigned int { ST_NONPHYSICAL = 1u, ST_NOROOT = 2u, ST_TIMEOUT = 4u, ST_NEGATIVE_DEPTH = 8u, ST_BOUNDS = 16u };

// Index guard of the bounds-checked build (compiled with LBMH_CHECK_BOUNDS):
// an index outside [0, n) sets ST_BOUNDS in *st and is clamped into range, so
// a wrong index shows up as a status bit (and wrong values), never as a
// memory fault.  In other builds it is the identity and costs nothing.
template <class I>
__device__ __forceinline__ I chk(I i, long long n, unsigned int* st) {
#ifdef LBMH_CHECK_BOUNDS
  if ((long long)i < 0 || (long long)i >= n) {
    if (st) atomicOr(st, ST_BOUNDS);
    return (long long)i < 0 ? I(0) : I(n - 1);
  }
#else
  (void)n;
  (void)st;
#endif
  return i;
}

// Coefficients of one step, computed identically by every thread from the
// control slot: dt (2.21), lambda = dx/dt, alpha_j = abar_j + eps, and the
// equilibrium weights a_k of (2.5)/(2.20).
struct StepCoef {
  double dt, lam, alpha[2], a0, aj[2];
  int active;
};

__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

inline double bits_to_host(unsigned long long b) {
  union {
    unsigned long long u;
    double d;
  } v;
  v.u = b;
  return v.d;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* slot, double v) {
  // max of non-negative doubles == max of their bit patterns; NaN (bit pattern
  // above +inf) wins, which keeps a blown-up state visible
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

template <int D>
__device__ __forceinline__ StepCoef step_coef(const DevParams& P, const Ctl* ctl, int slot) {
  StepCoef c;
  double ab0 = bits_to_double(ctl->amax[slot][0]);
  double ab1 = D == 2 ? bits_to_double(ctl->amax[slot][1]) : 0.0;
  double t = ctl->t[slot];
  c.active = !(P.T > 0.0 && t >= P.T) && !(P.max_steps > 0 && ctl->nsteps[slot] >= P.max_steps);
  double asum = D == 2 ? ab0 + ab1 : ab0;
  c.dt = P.cfl * P.dx / asum;
  c.lam = P.dx / c.dt;
  c.alpha[0] = ab0 + P.eps;
  c.alpha[1] = D == 2 ? ab1 + P.eps : 0.0;
  double alsum = D == 2 ? c.alpha[0] + c.alpha[1] : c.alpha[0];
  c.a0 = 1.0 - alsum / c.lam;
  c.aj[0] = c.alpha[0] / (2.0 * c.lam);
  c.aj[1] = c.alpha[1] / (2.0 * c.lam);
  return c;
}

// Block 0 advances the control block: slot+1 receives t, step count and
// parity; slot+2 is cleared for the step after next.
template <int D>
__device__ __forceinline__ void advance_ctl(Ctl* ctl, int slot, const StepCoef& c) {
  int s1 = (slot + 1) % 3, s2 = (slot + 2) % 3;
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
  }
  ctl->amax[s2][0] = 0ull;
  ctl->amax[s2][1] = 0ull;
}

// offset of node (i, j) inside a distribution plane
__host__ __device__ __forceinline__ long long cell(const DevParams& P, int i, int j) {
  return (long long)j * P.pitch + i + XPAD;
}

// index of a ghost coordinate e in [-3, n+3) mapped into [0, n): periodic
// wraps, outflow clamps (every read of f^n outside the domain is a read of the
// nearest interior node, or of the wrapped node)
__device__ __forceinline__ int map_index(int e, int n, int bc_lo, int bc_hi) {
  if (e < 0) return bc_lo == BC_PERIODIC ? (e % n + n) % n : (bc_lo == BC_REFLECT ? -1 - e : 0);
  if (e >= n) return bc_hi == BC_PERIODIC ? e % n : (bc_hi == BC_REFLECT ? 2 * n - 1 - e : n - 1);
  return e;
}

// boundary type across which coordinate e lies (-1 inside [0, n))
__device__ __forceinline__ int ghost_side(int e, int n, int bc_lo, int bc_hi) {
  return e < 0 ? bc_lo : (e >= n ? bc_hi : -1);
}

// index of the position of extended coordinate e: a periodic or outflow ghost
// sits where the node it copies sits, a reflecting ghost at its own position
__device__ __forceinline__ int pos_index(int e, int n, int bc_lo, int bc_hi) {
  return ghost_side(e, n, bc_lo, bc_hi) == BC_REFLECT ? e : map_index(e, n, bc_lo, bc_hi);
}

}  // namespace lbmh
