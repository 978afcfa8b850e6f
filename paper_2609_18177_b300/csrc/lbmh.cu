// Host side of the lbmh C ABI: validation, device memory, step launches and
// the template dispatch over (system, dimension, precision).
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/lbmh.h"
#include "common.cuh"
#include "fused.cuh"
#include "host_util.h"
#include "physics.cuh"
#include "state.cuh"
#include "lbm3d.cuh"
#include "lbm3d_fused.cuh"
#include "unfused.cuh"

using namespace lbmh;

namespace {

struct Ops;

}  // namespace

struct lbmh_handle {
  lbmh_problem prob;
  DevParams P;
  int m, Q, dim, sys, prec;
  int kernel;               // LBMH_KERNEL_FUSED or LBMH_KERNEL_UNFUSED
  size_t elem;              // sizeof(real)
  long long plane;          // ny * pitch
  cudaStream_t stream;
  void* fbuf[2];
  void** dbuf;              // device copy of fbuf
  void* Ue;                 // unfused scratch: U_ext [m][ey][ex] (3D: two copies, by f parity)
  bool u3_valid;            // 3D: the U copy of the current f holds its moments (interior)
  bool idx64_3d;            // 3D: 64-bit offsets in the collision kernel even where int offsets fit
  void* nue;                // nu_ext
  void* ome;                // omega_ext
  ExtGeom G;
  double* partials;         // per-block FP64 sums of the last step
  int nblocks;              // blocks writing partials in the last step
  int max_blocks;
  Ctl* ctl;
  double* Utmp;             // FP64 staging, allocated on first use
  size_t utmp_bytes;
  long long launched;       // step launches since set_state
  bool has_state;
  long long device_bytes;
  const Ops* ops;
  FusedPlan fp;
  // runs of kGraphSteps launches replayed as one CUDA graph (captured on a
  // private stream, keyed by the end time T the launches carry)
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;
  double graph_T;
  bool graph_failed;
  int halo_lo, halo_hi;     // slab of a lattice decomposed along y: halo rows below / above the window
  std::string err;
};

namespace {

// message of the last failure that had no handle (lbmh_create, lbmh_step_static),
// kept per host thread so that concurrent callers do not read each other's
thread_local std::string g_create_error;

int fail(lbmh_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(lbmh_handle* h, cudaError_t e, const char* what) {
  return fail(h, LBMH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int set_state_impl(lbmh_handle* h, const double* U, int on_device, const double* abar);
size_t halo_bytes(const lbmh_handle* h);
__global__ void k_set_bound(Ctl* ctl, int slot, unsigned long long b0, unsigned long long b1);

#define CK(h, call)                                    \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)


// ---------------------------------------------------------------------------
// per-(system, dimension, precision) operations
// ---------------------------------------------------------------------------

int ensure_scratch(lbmh_handle* h);
void free_scratch(lbmh_handle* h);

struct Ops {
  int (*launch_step)(lbmh_handle*, int slot, double T);
  int (*launch_unfused_diag)(lbmh_handle*, int slot);  // K0..K2 only
  int (*init)(lbmh_handle*, const double* U0dev, bool bound_given);  // bound_given: ctl->ainit is set
  int (*moments)(lbmh_handle*, int slot, double* Udev);
  int (*get_f)(lbmh_handle*, int slot, double* dev);
  int (*set_f)(lbmh_handle*, const double* dev);
  int (*omega_extract)(lbmh_handle*, double* dev);
  int (*setup_fused)(lbmh_handle*);
  bool has_fused;
};

template <int SYS, int D, class R>
struct Impl {
  static constexpr int M = Fields<SYS, D>::M, Q = Fields<SYS, D>::Q;

  static void fill_pads(lbmh_handle* h, R* f) {
    long long n = (long long)h->P.ny * Q * M * 2 * NGHOST;
    k_fill_pads<R><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, Q * M, f, h->ctl);
  }

  static int unfused_front(lbmh_handle* h, int slot, const DevParams& P) {
    long long next = (long long)h->G.ex * h->G.ey * h->G.ez;
    unsigned nb = blocks_for(next);
    R* const* buf = (R* const*)h->dbuf;
    k_moments_ext<SYS, D, R><<<nb, kBlock, 0, h->stream>>>(P, buf, h->ctl, slot, h->G, (R*)h->Ue);
    k_indicator<SYS, D, R><<<nb, kBlock, 0, h->stream>>>(P, h->ctl, slot, h->G, (const R*)h->Ue, (R*)h->nue);
    k_omega<D, R><<<nb, kBlock, 0, h->stream>>>(P, h->ctl, slot, h->G, (const R*)h->nue, (R*)h->ome);
    return LBMH_OK;
  }

  static int launch_step(lbmh_handle* h, int slot, double T) {
    DevParams P = h->P;
    P.T = T;
    if (h->kernel == LBMH_KERNEL_FUSED) {
      h->nblocks = fused_launch<SYS, D, R>(h->fp, P, (R* const*)h->dbuf, h->ctl, slot, h->partials, h->stream);
    } else {
      unfused_front(h, slot, P);
      long long nn = (long long)P.nx * P.ny;
      unsigned nb = blocks_for(nn);
      k_collide_stream<SYS, D, R><<<nb, kBlock, 0, h->stream>>>(P, (R* const*)h->dbuf, h->ctl, slot, h->G,
                                                                (const R*)h->Ue, (const R*)h->ome, h->partials);
      h->nblocks = (int)nb;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    return LBMH_OK;
  }

  static int launch_unfused_diag(lbmh_handle* h, int slot) {
    DevParams P = h->P;
    P.T = 0.0;
    unfused_front(h, slot, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostic launch");
    return LBMH_OK;
  }

  static int init(lbmh_handle* h, const double* U0dev, bool bound_given) {
    long long nn = (long long)h->P.nx * h->P.ny;
    unsigned nb = reduce_blocks_for(nn);
    if (!bound_given) k_init_speed<SYS, D><<<nb, kBlock, 0, h->stream>>>(h->P, U0dev, h->ctl);
    k_init_eq<SYS, D, R><<<nb, kBlock, 0, h->stream>>>(h->P, U0dev, (R*)h->fbuf[0], h->ctl);
    fill_pads(h, (R*)h->fbuf[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "init launch");
    return LBMH_OK;
  }

  static int moments(lbmh_handle* h, int slot, double* Udev) {
    long long nn = (long long)h->P.nx * h->P.ny;
    k_moments<M, Q, R><<<blocks_for(nn), kBlock, 0, h->stream>>>(h->P, (R* const*)h->dbuf, h->ctl, slot, Udev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "moments launch");
    return LBMH_OK;
  }

  static int get_f(lbmh_handle* h, int slot, double* dev) {
    long long n = (long long)h->P.nx * h->P.ny * Q * M;
    k_get_f<R><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, Q * M, (R* const*)h->dbuf, h->ctl, slot, dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "get_f launch");
    return LBMH_OK;
  }

  static int set_f(lbmh_handle* h, const double* dev) {
    long long n = (long long)h->P.nx * h->P.ny * Q * M;
    k_set_f<R><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, Q * M, (R*)h->fbuf[0], dev, h->ctl);
    fill_pads(h, (R*)h->fbuf[0]);
    k_speed_of_f<SYS, D, R><<<reduce_blocks_for((long long)h->P.nx * h->P.ny), kBlock, 0, h->stream>>>(
        h->P, (R* const*)h->dbuf, h->ctl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "set_f launch");
    return LBMH_OK;
  }

  static int omega_extract(lbmh_handle* h, double* dev) {
    long long nn = (long long)h->P.nx * h->P.ny;
    k_extract_interior<R><<<blocks_for(nn), kBlock, 0, h->stream>>>(h->P, h->G, (const R*)h->ome, dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "omega launch");
    return LBMH_OK;
  }

  static int setup_fused(lbmh_handle* h) { return fused_setup<SYS, D, R>(h->fp, h->P, h->fbuf); }

  static const Ops* ops() {
    static const Ops o = {launch_step, launch_unfused_diag, init, moments, get_f, set_f, omega_extract, setup_fused,
                          fused_available<SYS, D, R>()};
    return &o;
  }
};

// 3D (D3Q7) operations: the four-kernel path of lbm3d.cuh; the row-wise
// kernels (moments, checkpoints) are shared with 1D/2D (rows = z * ny + y)
template <int SYS, class R>
struct Impl3 {
  static constexpr int M = Fields3<SYS>::M, Q = 7;

  static ExtGeom3 geom(const lbmh_handle* h) { return ExtGeom3{h->G.ex, h->G.ey, h->G.ez, ext_pitch3(h->G.ex)}; }

  static int launch_step(lbmh_handle* h, int slot, double T) {
    DevParams P = h->P;
    P.T = T;
    const ExtGeom3 G = geom(h);
    const dim3 ge = grid3_ext(G.ex, G.ey, G.ez), gn = grid3_nodes(P.nx, P.ny3, P.nz3);
    R* const* buf = (R* const*)h->dbuf;
    if (h->u3_valid) {  // the previous step's collision wrote the interior of U
      const long long ng = (long long)G.ex * G.ey * G.ez - (long long)P.nx * P.ny3 * P.nz3;
      k3_ghost_fill<SYS, R><<<(unsigned)((ng + kBlock3 - 1) / kBlock3), kBlock3, 0, h->stream>>>(P, h->ctl, slot, G,
                                                                                               (R*)h->Ue);
    } else {
      k3_moments_ext<SYS, R><<<ge, kBlock3, 0, h->stream>>>(P, buf, h->ctl, slot, G, (R*)h->Ue);
    }
    if (h->kernel == LBMH_KERNEL_FUSED) {  // indicator, omega, collision and streaming in one pass
      using T3 = Tile3F<SYS, R>;
      const int zc = h->fp.band;
      const dim3 gf = grid3_fused(P.nx, P.ny3, P.nz3, T3::TY, zc);
      k3_fused<SYS, R><<<gf, T3::threads, h->fp.smem, h->stream>>>(h->fp.tu3[0], h->fp.tu3[1], h->fp.tf3[0],
                                                                   h->fp.tf3[1], P, buf, h->ctl, slot, G, (R*)h->Ue,
                                                                   h->partials, zc);
      h->u3_valid = true;
      h->nblocks = (int)(gf.x * gf.y * gf.z) * (T3::threads / 32);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(h, e, "3D fused step launch");
      return LBMH_OK;
    }
    k3_indicator<SYS, R><<<ge, kBlock3, 0, h->stream>>>(P, h->ctl, slot, G, (const R*)h->Ue, (R*)h->nue);
    k3_omega<R><<<grid3_omega(G.ex, G.ey, G.ez), kBlock3, 0, h->stream>>>(P, h->ctl, slot, G, (const R*)h->nue,
                                                                          (R*)h->ome);
    if (!h->idx64_3d && k3_offsets_fit_int(P, M, G.size()))
      k3_collide_stream<SYS, R, int><<<gn, kBlock3, 0, h->stream>>>(P, buf, h->ctl, slot, G, (R*)h->Ue,
                                                                    (const R*)h->ome, h->partials);
    else
      k3_collide_stream<SYS, R, long long><<<gn, kBlock3, 0, h->stream>>>(P, buf, h->ctl, slot, G, (R*)h->Ue,
                                                                          (const R*)h->ome, h->partials);
    h->u3_valid = true;
    h->nblocks = (int)(gn.x * gn.y * gn.z) * (kLanes3 / 32);  // one partial slot per warp
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "3D step launch");
    return LBMH_OK;
  }

  static int launch_unfused_diag(lbmh_handle* h, int) {
    return fail(h, LBMH_ERR_UNSUPPORTED, "the omega diagnostic is not provided for 3D lattices");
  }

  static int init(lbmh_handle* h, const double* U0dev, bool bound_given) {
    const long long nn = (long long)h->P.nx * h->P.ny;
    const unsigned nb = reduce_blocks_for(nn);
    if (!bound_given) k3_init_speed<SYS><<<nb, kBlock, 0, h->stream>>>(h->P, U0dev, h->ctl);
    k3_init_eq<SYS, R><<<nb, kBlock, 0, h->stream>>>(h->P, U0dev, (R*)h->fbuf[0], h->ctl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "3D init launch");
    return LBMH_OK;
  }

  static int moments(lbmh_handle* h, int slot, double* Udev) {
    const long long nn = (long long)h->P.nx * h->P.ny;
    k_moments<M, Q, R><<<blocks_for(nn), kBlock, 0, h->stream>>>(h->P, (R* const*)h->dbuf, h->ctl, slot, Udev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "moments launch");
    return LBMH_OK;
  }

  static int get_f(lbmh_handle* h, int slot, double* dev) {
    const long long n = (long long)h->P.nx * h->P.ny * Q * M;
    k_get_f<R><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, Q * M, (R* const*)h->dbuf, h->ctl, slot, dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "get_f launch");
    return LBMH_OK;
  }

  static int set_f(lbmh_handle* h, const double* dev) {
    const long long n = (long long)h->P.nx * h->P.ny * Q * M;
    k_set_f<R><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, Q * M, (R*)h->fbuf[0], dev, h->ctl);
    k3_speed_of_f<SYS, R><<<reduce_blocks_for((long long)h->P.nx * h->P.ny), kBlock, 0, h->stream>>>(
        h->P, (R* const*)h->dbuf, h->ctl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "set_f launch");
    return LBMH_OK;
  }

  static int omega_extract(lbmh_handle* h, double*) {
    return fail(h, LBMH_ERR_UNSUPPORTED, "the omega diagnostic is not provided for 3D lattices");
  }

  // the fused step's shared memory, z chunk (planes a block marches; at least
  // 8; LBMH_3D_ZCHUNK overrides it for tuning runs) and partial-sum slots
  static int setup_fused(lbmh_handle* h) {
    using L = Smem3F<SYS, R>;
    using T3 = Tile3F<SYS, R>;
    auto kern = k3_fused<SYS, R>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::total) != cudaSuccess)
      return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T3::threads, L::total) != cudaSuccess ||
        per_sm < 1)
      return -1;
    int zc = 32;
    const char* e = getenv("LBMH_3D_ZCHUNK");
    if (e && atoi(e) >= 8) zc = atoi(e);
    // the U boxes read the ghost-extended copies: allocated here (the two U
    // copies only), then described to the TMA unit
    if (ensure_scratch(h) != LBMH_OK) return -1;
    if (k3f_encode_maps<SYS, R>(h->fp, h->P, geom(h), h->Ue, h->fbuf) != 0) {
      free_scratch(h);
      return -1;
    }
    h->fp.smem = (int)L::total;
    h->fp.band = zc;
    const dim3 g = grid3_fused(h->P.nx, h->P.ny3, h->P.nz3, T3::TY, zc);
    h->fp.blocks = (int)(g.x * g.y * g.z) * (T3::threads / 32);
    return 0;
  }

  static const Ops* ops() {
    static const Ops o = {launch_step, launch_unfused_diag, init, moments, get_f, set_f, omega_extract, setup_fused,
                          true};
    return &o;
  }
};

template <class R>
const Ops* pick_dim(int sys, int dim) {
  if (dim == 3) {
    switch (sys) {
      case SYS_ADV: return Impl3<SYS_ADV, R>::ops();
      case SYS_EULER: return Impl3<SYS_EULER, R>::ops();
      case SYS_REACT: return Impl3<SYS_REACT, R>::ops();
    }
    return nullptr;
  }
#define PICK(S)                                        \
  case S:                                              \
    return dim == 1 ? Impl<S, 1, R>::ops() : Impl<S, 2, R>::ops();
  switch (sys) {
    PICK(SYS_ADV)
    PICK(SYS_EULER)
    PICK(SYS_SWE)
    PICK(SYS_REACT)
  }
#undef PICK
  return nullptr;
}

const Ops* pick_ops(int sys, int dim, int prec) {
  return prec == LBMH_FP32 ? pick_dim<float>(sys, dim) : pick_dim<double>(sys, dim);
}

void free_handle(lbmh_handle* h) {
  if (!h) return;
  cudaFree(h->fbuf[0]);
  cudaFree(h->fbuf[1]);
  cudaFree(h->dbuf);
  cudaFree(h->Ue);
  cudaFree(h->nue);
  cudaFree(h->ome);
  cudaFree(h->partials);
  cudaFree(h->ctl);
  cudaFree(h->Utmp);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

// device staging for host transfers and FP64 conversions, grown on demand
int ensure_utmp(lbmh_handle* h, size_t bytes) {
  if (h->utmp_bytes >= bytes) return LBMH_OK;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->Utmp);
  h->device_bytes -= (long long)h->utmp_bytes;
  h->Utmp = nullptr;
  h->utmp_bytes = 0;
  if (cudaMalloc((void**)&h->Utmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, LBMH_ERR_OOM, "device allocation of the staging buffer failed");
  }
  h->utmp_bytes = bytes;
  h->device_bytes += (long long)bytes;
  return LBMH_OK;
}

// releases the ghost-extended scratch (ensure_scratch allocates it again)
void free_scratch(lbmh_handle* h) {
  long long next = (long long)(h->dim == 3 ? ext_pitch3(h->G.ex) : h->G.ex) * h->G.ey * h->G.ez;
  size_t b1 = (size_t)next * h->m * h->elem * (h->dim == 3 ? 2 : 1), b2 = (size_t)next * h->elem;
  if (h->Ue) h->device_bytes -= (long long)b1;
  if (h->nue) h->device_bytes -= (long long)b2;
  if (h->ome) h->device_bytes -= (long long)b2;
  cudaFree(h->Ue);
  cudaFree(h->nue);
  cudaFree(h->ome);
  h->Ue = h->nue = h->ome = nullptr;
}

// ghost-extended scratch of the unfused path (also used by lbmh_omega)
int ensure_scratch(lbmh_handle* h) {
  if (h->Ue) return LBMH_OK;
  // 3D rows are padded to ext_pitch3 (16-byte row starts for the TMA boxes)
  long long next = (long long)(h->dim == 3 ? ext_pitch3(h->G.ex) : h->G.ex) * h->G.ey * h->G.ez;
  size_t b1 = (size_t)next * h->m * h->elem * (h->dim == 3 ? 2 : 1), b2 = (size_t)next * h->elem;
  // the fused 3D step keeps nu and omega on chip: only the two U copies
  const bool u_only = h->dim == 3 && h->kernel == LBMH_KERNEL_FUSED;
  if (u_only) b2 = 0;
  if (cudaMalloc(&h->Ue, b1) != cudaSuccess || (!u_only && cudaMalloc(&h->nue, b2) != cudaSuccess) ||
      (!u_only && cudaMalloc(&h->ome, b2) != cudaSuccess)) {
    cudaGetLastError();
    cudaFree(h->Ue);
    cudaFree(h->nue);
    cudaFree(h->ome);
    h->Ue = h->nue = h->ome = nullptr;
    return fail(h, LBMH_ERR_OOM, "device allocation of the unfused scratch failed");
  }
  h->device_bytes += (long long)(b1 + 2 * b2);
  return LBMH_OK;
}

int sync(lbmh_handle* h) {
  CK(h, cudaStreamSynchronize(h->stream));
  return LBMH_OK;
}

int current_slot(const lbmh_handle* h) { return (int)(h->launched % 3); }

// launches per graph: a multiple of 3 so that a replay starting at slot 0
// ends at slot 0 (the control block rotates through three slots)
constexpr int kGraphSteps = 24;

// capture kGraphSteps launches starting at slot 0 with end time T
int capture_steps(lbmh_handle* h, double T) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  cudaGraph_t g = nullptr;
  // a replay may follow any change of the distributions: its first step
  // computes the 3D moments in full
  const bool u3_before = h->u3_valid;
  h->u3_valid = false;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = LBMH_OK;
  if (e == cudaSuccess) {
    for (int s = 0; s < kGraphSteps && rc == LBMH_OK; s++) rc = h->ops->launch_step(h, s % 3, T);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  h->stream = user;
  if (e == cudaSuccess && rc == LBMH_OK) e = cudaGraphInstantiate(&h->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess || rc != LBMH_OK) {
    cudaGetLastError();
    h->graph = nullptr;
    h->u3_valid = u3_before;  // nothing ran
    h->graph_failed = true;  // fall back to single launches from now on
    h->err.clear();
    return LBMH_OK;
  }
  h->graph_T = T;
  return LBMH_OK;
}

// n step launches with end time T (0 = none): single launches up to the next
// multiple of 3, graph replays of kGraphSteps launches, single launches for
// the rest
int run_steps(lbmh_handle* h, int64_t n, double T) {
  int64_t s = 0;
  auto single = [&](int64_t upto) -> int {
    for (; s < upto; s++) {
      int rc = h->ops->launch_step(h, current_slot(h), T);
      if (rc) return rc;
      h->launched++;
    }
    return LBMH_OK;
  };
  if (n >= 2 * kGraphSteps && !h->graph_failed) {
    int rc = single((3 - current_slot(h)) % 3);
    if (rc) return rc;
    if (!h->graph || h->graph_T != T) {
      rc = capture_steps(h, T);
      if (rc) return rc;
    }
    if (h->graph) {
      for (; s + kGraphSteps <= n; s += kGraphSteps) {
        CK(h, cudaGraphLaunch(h->graph, h->stream));
        h->launched += kGraphSteps;
      }
    }
  }
  return single(n);
}

int read_ctl(lbmh_handle* h, Ctl* out) {
  CK(h, cudaMemcpyAsync(out, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  return sync(h);
}

}  // namespace

extern "C" {

#ifdef LBMH_CHECK_BOUNDS
const char* lbmh_version(void) { return "lbmh 0.2 sm_103a bounds-checked"; }
#else
const char* lbmh_version(void) { return "lbmh 0.2 sm_103a"; }
#endif

const char* lbmh_last_error(const lbmh_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

namespace {

// rows of a slab of a lattice decomposed along y, in its local lattice
struct SlabGeom {
  int halo_lo, halo_hi;  // halo rows below / above the rows it writes (0 or 3)
  int row0;              // global row of local row 0
};

int create_impl(const lbmh_problem* p, const SlabGeom* sg, lbmh_handle** out) {
  if (!out) return fail(nullptr, LBMH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  int rc = validate(p, why);
  if (rc) return fail(nullptr, rc, why);
  lbmh_handle* h = new lbmh_handle();
  memset(h->fbuf, 0, sizeof h->fbuf);
  h->dbuf = nullptr; h->Ue = h->nue = h->ome = nullptr; h->partials = nullptr; h->ctl = nullptr; h->Utmp = nullptr;
  h->cap_stream = nullptr; h->graph = nullptr; h->graph_T = 0.0; h->graph_failed = false; h->u3_valid = false;
  h->halo_lo = h->halo_hi = 0;
  {  // LBMH_3D_INDEX64=1 selects the 64-bit-offset collision kernel at any size (for tests)
    const char* e = getenv("LBMH_3D_INDEX64");
    h->idx64_3d = e && e[0] == '1';
  }
  h->prob = *p;
  h->dim = p->dim;
  h->sys = p->system;
  h->prec = p->precision;
  h->m = nfields(p->system, p->dim);
  h->Q = 2 * p->dim + 1;
  h->elem = p->precision == LBMH_FP32 ? sizeof(float) : sizeof(double);
  h->stream = (cudaStream_t)p->cuda_stream;
  h->ops = pick_ops(p->system, p->dim, p->precision);
  h->launched = 0;
  h->has_state = false;
  h->nblocks = 0;
  h->device_bytes = 0;
  h->P = make_devparams(p, padded_pitch(p->nx, h->elem));
  DevParams& P = h->P;
  h->plane = P.plane;
  apply_wait_hook(P);
  h->halo_lo = sg ? sg->halo_lo : 0;
  h->halo_hi = sg ? sg->halo_hi : 0;
  if (sg) {
    P.ywin0 = sg->halo_lo;
    P.ywin1 = P.ny - sg->halo_hi;
    P.row0 = sg->row0;
  }

  // 3D: the fused z-marching kernel by default in FP32 (256^3 Euler: 1.30
  // against 1.64 ms per step for the four-kernel path); in FP64, bound by the
  // FP64 pipe, the four-kernel path (25.7 against 33.7 ms) unless asked for
  const bool auto_fused3 = p->precision == LBMH_FP32;
  bool want_fused = p->dim == 3 ? (p->kernel == LBMH_KERNEL_FUSED || (p->kernel == LBMH_KERNEL_AUTO && auto_fused3))
                                : p->kernel != LBMH_KERNEL_UNFUSED;
  if (p->kernel == LBMH_KERNEL_FUSED && !h->ops->has_fused) {
    delete h;
    return fail(nullptr, LBMH_ERR_UNSUPPORTED, "no fused kernel for this system/dimension/precision");
  }
  h->kernel = (want_fused && h->ops->has_fused) ? LBMH_KERNEL_FUSED : LBMH_KERNEL_UNFUSED;
  if (h->kernel == LBMH_KERNEL_UNFUSED && needs_fused(p)) {
    delete h;
    return fail(nullptr, LBMH_ERR_UNSUPPORTED, "reflecting/inflow sides and the sponge need the fused kernel");
  }

  h->G.ex = P.nx + 2 * GH;
  h->G.gy = p->dim >= 2 ? GH : 0;
  h->G.ey = p->dim == 2 ? P.ny + 2 * GH : (p->dim == 3 ? P.ny3 + 2 * GH : 1);
  h->G.ez = p->dim == 3 ? P.nz3 + 2 * GH : 1;
  long long nn = (long long)P.nx * P.ny;
  size_t fbytes = (size_t)h->Q * h->m * P.plane * h->elem;
  h->max_blocks = (int)blocks_for(nn);
  if (p->dim == 3) {  // one partial slot per warp of the 3D collision kernel
    const dim3 g3 = grid3_nodes(P.nx, P.ny3, P.nz3);
    h->max_blocks = std::max(h->max_blocks, (int)(g3.x * g3.y * g3.z) * (kLanes3 / 32));
  }
  h->utmp_bytes = 0;
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    h->device_bytes += (long long)bytes;
    return true;
  };
  bool ok = alloc(&h->fbuf[0], fbytes) && alloc(&h->fbuf[1], fbytes);
  if (ok && h->kernel == LBMH_KERNEL_FUSED) {
    memset(&h->fp, 0, sizeof h->fp);
    if (h->ops->setup_fused(h) != 0) {
      cudaGetLastError();
      if (p->kernel == LBMH_KERNEL_FUSED || needs_fused(p)) {
        free_handle(h);
        return fail(nullptr, LBMH_ERR_CUDA, "fused kernel setup failed");
      }
      h->kernel = LBMH_KERNEL_UNFUSED;
    } else if (h->fp.blocks > h->max_blocks) {
      h->max_blocks = h->fp.blocks;
    }
  }
  ok = ok && alloc((void**)&h->dbuf, 2 * sizeof(void*)) &&
       alloc((void**)&h->partials, (size_t)h->max_blocks * h->m * sizeof(double)) &&
       alloc((void**)&h->ctl, sizeof(Ctl));
  if (ok && (h->kernel == LBMH_KERNEL_UNFUSED || h->dim == 3) && ensure_scratch(h) != LBMH_OK) ok = false;
  if (!ok) {
    free_handle(h);
    return fail(nullptr, LBMH_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpy(h->dbuf, h->fbuf, 2 * sizeof(void*), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->partials, 0, (size_t)h->max_blocks * h->m * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->ctl, 0, sizeof(Ctl));
  if (e != cudaSuccess) {
    std::string msg = std::string("setup: ") + cudaGetErrorString(e);
    free_handle(h);
    return fail(nullptr, LBMH_ERR_CUDA, msg);
  }
  *out = h;
  return LBMH_OK;
}

}  // namespace

extern "C" {

int lbmh_create(const lbmh_problem* p, lbmh_handle** out) { return create_impl(p, nullptr, out); }

int lbmh_destroy(lbmh_handle* h) {
  if (!h) return LBMH_OK;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
  return LBMH_OK;
}

int lbmh_set_state(lbmh_handle* h, const double* U, int on_device) { return set_state_impl(h, U, on_device, nullptr); }

int lbmh_set_state_bound(lbmh_handle* h, const double* U, int on_device, const double* abar) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!abar) return fail(h, LBMH_ERR_INVALID_ARG, "abar is NULL");
  if (h->dim == 3) return fail(h, LBMH_ERR_UNSUPPORTED, "lbmh_set_state_bound serves 1D and 2D lattices");
  for (int j = 0; j < h->dim; j++)
    if (!(abar[j] > 0.0) || !std::isfinite(abar[j])) return fail(h, LBMH_ERR_INVALID_ARG, "abar must be positive and finite");
  return set_state_impl(h, U, on_device, abar);
}

}  // extern "C"

namespace {

// f := f^eq(U) (Eq. 2.20) with alpha^0, lambda^0 from U's speed bound, or from
// abar when given (then already in host memory: staged by the copy below)
int set_state_impl(lbmh_handle* h, const double* U, int on_device, const double* abar) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!U) return fail(h, LBMH_ERR_INVALID_ARG, "U is NULL");
  h->err.clear();
  long long nn = (long long)h->P.nx * h->P.ny;
  size_t bytes = (size_t)nn * h->m * sizeof(double);
  const double* src = U;
  if (!on_device) {
    int rc0 = ensure_utmp(h, bytes);
    if (rc0) return rc0;
    CK(h, cudaMemcpyAsync(h->Utmp, U, bytes, cudaMemcpyHostToDevice, h->stream));
    src = h->Utmp;
  }
  CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
  if (abar)
    CK(h, cudaMemcpyAsync((char*)h->ctl + offsetof(Ctl, ainit), abar, h->dim * sizeof(double), cudaMemcpyHostToDevice,
                          h->stream));
  h->u3_valid = false;
  int rc = h->ops->init(h, src, abar != nullptr);
  if (rc) return rc;
  if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
  h->launched = 0;
  h->has_state = true;
  h->nblocks = 0;
  return LBMH_OK;
}

}  // namespace

extern "C" {

int lbmh_step(lbmh_handle* h, int64_t n) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state: call lbmh_set_state first");
  if (n < 0) return fail(h, LBMH_ERR_INVALID_ARG, "negative step count");
  h->err.clear();
  return run_steps(h, n, 0.0);
}

int lbmh_advance_to(lbmh_handle* h, double T, int64_t max_steps) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state: call lbmh_set_state first");
  if (!(T > 0.0) || max_steps < 0) return fail(h, LBMH_ERR_INVALID_ARG, "T must be positive");
  h->err.clear();
  int64_t done = 0;
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  long long start = c.nsteps[current_slot(h)];
  while (done < max_steps) {
    int slot = current_slot(h);
    double t = c.t[slot];
    if (t >= T) break;
    double ab = bits_to_host(c.amax[slot][0]) + (h->dim >= 2 ? bits_to_host(c.amax[slot][1]) : 0.0) +
                (h->dim == 3 ? bits_to_host(c.amax_z[slot]) : 0.0);
    double dt_est = h->P.cfl * h->P.dx / ab;
    int64_t est = (int64_t)((T - t) / dt_est) + 1;
    int64_t chunk = est < 8 ? 8 : (est > 256 ? 256 : est);
    if (chunk > max_steps - done) chunk = max_steps - done;
    rc = run_steps(h, chunk, T);
    if (rc) return rc;
    rc = read_ctl(h, &c);
    if (rc) return rc;
    done = c.nsteps[current_slot(h)] - start;
    if (c.status & ST_NONPHYSICAL) break;
  }
  return LBMH_OK;
}

int lbmh_moments(lbmh_handle* h, double* U_out, int on_device, double* t, int64_t* steps) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  if (!U_out) return fail(h, LBMH_ERR_INVALID_ARG, "U_out is NULL");
  long long nn = (long long)h->P.nx * h->P.ny;
  size_t bytes = (size_t)nn * h->m * sizeof(double);
  int slot = current_slot(h);
  if (!on_device) {
    int rc0 = ensure_utmp(h, bytes);
    if (rc0) return rc0;
  }
  int rc = h->ops->moments(h, slot, on_device ? U_out : h->Utmp);
  if (rc) return rc;
  if (!on_device) CK(h, cudaMemcpyAsync(U_out, h->Utmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  Ctl c;
  rc = read_ctl(h, &c);
  if (rc) return rc;
  if (t) *t = c.t[slot];
  if (steps) *steps = c.nsteps[slot];
  if (c.status & ST_BOUNDS) return fail(h, LBMH_ERR_BOUNDS, "an index left its array (bounds-checked build)");
  if (c.status & ST_TIMEOUT) return fail(h, LBMH_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (c.status & ST_NONPHYSICAL) return fail(h, LBMH_ERR_NONPHYSICAL, "a step produced a non-physical state");
  return LBMH_OK;
}

int lbmh_get_f(lbmh_handle* h, double* f_out, int on_device, double* t, int64_t* steps) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  if (!f_out) return fail(h, LBMH_ERR_INVALID_ARG, "f_out is NULL");
  long long n = (long long)h->P.nx * h->P.ny * h->Q * h->m;
  int slot = current_slot(h);
  if (!on_device) {
    int rc0 = ensure_utmp(h, (size_t)n * sizeof(double));
    if (rc0) return rc0;
  }
  int rc = h->ops->get_f(h, slot, on_device ? f_out : h->Utmp);
  if (rc) return rc;
  if (!on_device) CK(h, cudaMemcpyAsync(f_out, h->Utmp, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  Ctl c;
  rc = read_ctl(h, &c);
  if (rc) return rc;
  if (t) *t = c.t[slot];
  if (steps) *steps = c.nsteps[slot];
  return LBMH_OK;
}

int lbmh_set_f(lbmh_handle* h, const double* f_in, int on_device, double t, int64_t steps) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!f_in) return fail(h, LBMH_ERR_INVALID_ARG, "f_in is NULL");
  long long n = (long long)h->P.nx * h->P.ny * h->Q * h->m;
  const double* src = f_in;
  if (!on_device) {
    int rc0 = ensure_utmp(h, (size_t)n * sizeof(double));
    if (rc0) return rc0;
    CK(h, cudaMemcpyAsync(h->Utmp, f_in, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    src = h->Utmp;
  }
  Ctl c;
  memset(&c, 0, sizeof c);
  c.t[0] = t;
  c.nsteps[0] = steps;
  CK(h, cudaMemcpyAsync(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice, h->stream));
  h->u3_valid = false;
  int rc = h->ops->set_f(h, src);
  if (rc) return rc;
  rc = sync(h);
  if (rc) return rc;
  h->launched = 0;
  h->has_state = true;
  return LBMH_OK;
}

int lbmh_omega(lbmh_handle* h, double* out, int on_device) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  if (!out) return fail(h, LBMH_ERR_INVALID_ARG, "out is NULL");
  long long nn = (long long)h->P.nx * h->P.ny;
  int slot = current_slot(h);
  int rc = ensure_scratch(h);
  if (rc) return rc;
  if (!on_device) {
    rc = ensure_utmp(h, (size_t)nn * sizeof(double));
    if (rc) return rc;
  }
  rc = h->ops->launch_unfused_diag(h, slot);
  if (rc) return rc;
  rc = h->ops->omega_extract(h, on_device ? out : h->Utmp);
  if (rc) return rc;
  if (!on_device) CK(h, cudaMemcpyAsync(out, h->Utmp, (size_t)nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return sync(h);
}

int lbmh_get_info(lbmh_handle* h, lbmh_info* out) {
  if (!h || !out) return LBMH_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  out->m = h->m;
  out->Q = h->Q;
  out->kernel = h->kernel;
  out->device_bytes = h->device_bytes;
  if (h->halo_lo || h->halo_hi) {
    out->halo_bytes = (int64_t)halo_bytes(h);
    out->halo_rows[0] = h->halo_lo;
    out->halo_rows[1] = h->halo_hi;
    out->row0 = h->P.row0;
  }
  if (!h->has_state) return LBMH_OK;
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  int slot = current_slot(h);
  out->t = c.t[slot];
  out->steps = c.nsteps[slot];
  out->abar[0] = bits_to_host(c.amax[slot][0]);
  out->abar[1] = bits_to_host(c.amax[slot][1]);
  out->abar_z = h->dim == 3 ? bits_to_host(c.amax_z[slot]) : 0.0;
  out->last_dt = c.last_dt;
  out->last_lambda = c.last_lambda;
  out->status = c.status;
  if (h->nblocks > 0) {
    std::vector<double> part((size_t)h->nblocks * h->m);
    CK(h, cudaMemcpy(part.data(), h->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int b = 0; b < h->nblocks; b++)
      for (int c2 = 0; c2 < h->m && c2 < 8; c2++) out->sum_U[c2] += part[(size_t)b * h->m + c2];
  }
  return LBMH_OK;
}

// ---------------------------------------------------------------------------
// Slabs: one 2D lattice decomposed along y into row ranges, one handle per
// range (one per GPU).  A slab stores its rows plus three halo rows on each
// side that borders another slab, and writes only its own rows; per step the
// caller (1) takes the maximum of the slabs' speed bounds (Eq. 2.19: the
// maximum over x is global), (2) steps every slab, (3) copies each slab's
// three outermost rows into the neighbour's halo.  Node positions use global
// rows and every node runs the single-lattice arithmetic, so the slabs hold
// the bits of the whole lattice.
// ---------------------------------------------------------------------------

int lbmh_create_slab(const lbmh_problem* g, int row_begin, int row_end, lbmh_handle** out) {
  if (!out) return fail(nullptr, LBMH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  int rc = validate(g, why);
  if (rc) return fail(nullptr, rc, why);
  if (g->dim != 2) return fail(nullptr, LBMH_ERR_UNSUPPORTED, "slabs decompose 2D lattices");
  if (g->kernel == LBMH_KERNEL_UNFUSED) return fail(nullptr, LBMH_ERR_UNSUPPORTED, "slabs run the fused kernel");
  if (row_begin < 0 || row_end > g->ny || row_end - row_begin < 3)
    return fail(nullptr, LBMH_ERR_INVALID_ARG, "a slab needs rows [row_begin, row_end) within the lattice, at least 3");
  const bool whole = row_begin == 0 && row_end == g->ny;
  const bool periodic = g->bc[2] == LBMH_BC_PERIODIC;
  SlabGeom sg;
  sg.halo_lo = !whole && (row_begin > 0 || periodic) ? 3 : 0;
  sg.halo_hi = !whole && (row_end < g->ny || periodic) ? 3 : 0;
  sg.row0 = row_begin - sg.halo_lo;
  lbmh_problem lp = *g;
  const double dy = (g->y1 - g->y0) / g->ny;
  lp.ny = row_end - row_begin + sg.halo_lo + sg.halo_hi;
  lp.y1 = g->y0 + lp.ny * dy;  // positions come from global rows: y0 stays the lattice's
  if (sg.halo_lo) lp.bc[2] = LBMH_BC_OUTFLOW;  // never read: the rows beyond a halo are not needed
  if (sg.halo_hi) lp.bc[3] = LBMH_BC_OUTFLOW;
  lp.kernel = LBMH_KERNEL_FUSED;
  return create_impl(&lp, &sg, out);
}

int lbmh_state_speed_bound(lbmh_handle* h, const double* U, int on_device, double* abar_out) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!U || !abar_out) return fail(h, LBMH_ERR_INVALID_ARG, "U and abar_out must not be NULL");
  if (h->dim == 3) return fail(h, LBMH_ERR_UNSUPPORTED, "lbmh_state_speed_bound serves 1D and 2D lattices");
  h->err.clear();
  const long long nn = (long long)h->P.nx * h->P.ny;
  const size_t bytes = (size_t)nn * h->m * sizeof(double);
  const double* src = U;
  if (!on_device) {
    int rc0 = ensure_utmp(h, bytes);
    if (rc0) return rc0;
    CK(h, cudaMemcpyAsync(h->Utmp, U, bytes, cudaMemcpyHostToDevice, h->stream));
    src = h->Utmp;
  }
  // ctl->ainit is read only while a state is initialised, so it serves as the
  // reduction target here
  CK(h, cudaMemsetAsync((char*)h->ctl + offsetof(Ctl, ainit), 0, 2 * sizeof(double), h->stream));
  const unsigned nb = reduce_blocks_for(nn);
  switch (h->sys * 2 + (h->dim - 1)) {
    case SYS_ADV * 2 + 0: k_init_speed<SYS_ADV, 1><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_ADV * 2 + 1: k_init_speed<SYS_ADV, 2><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_EULER * 2 + 0: k_init_speed<SYS_EULER, 1><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_EULER * 2 + 1: k_init_speed<SYS_EULER, 2><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_SWE * 2 + 0: k_init_speed<SYS_SWE, 1><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_SWE * 2 + 1: k_init_speed<SYS_SWE, 2><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_REACT * 2 + 0: k_init_speed<SYS_REACT, 1><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    case SYS_REACT * 2 + 1: k_init_speed<SYS_REACT, 2><<<nb, kBlock, 0, h->stream>>>(h->P, src, h->ctl); break;
    default: return fail(h, LBMH_ERR_INVALID_ARG, "unknown system");
  }
  CK(h, cudaGetLastError());
  double a[2] = {0.0, 0.0};
  CK(h, cudaMemcpyAsync(a, (char*)h->ctl + offsetof(Ctl, ainit), sizeof a, cudaMemcpyDeviceToHost, h->stream));
  int rc = sync(h);
  if (rc) return rc;
  for (int j = 0; j < h->dim; j++) abar_out[j] = a[j];
  return LBMH_OK;
}

int lbmh_get_speed_bound(lbmh_handle* h, double* abar_out) {
  if (!h || !abar_out) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  const int slot = current_slot(h);
  abar_out[0] = bits_to_host(c.amax[slot][0]);
  if (h->dim >= 2) abar_out[1] = bits_to_host(c.amax[slot][1]);
  if (h->dim == 3) abar_out[2] = bits_to_host(c.amax_z[slot]);
  return LBMH_OK;
}

int lbmh_set_speed_bound(lbmh_handle* h, const double* abar) {
  if (!h || !abar) return LBMH_ERR_INVALID_ARG;
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  if (h->dim == 3) return fail(h, LBMH_ERR_UNSUPPORTED, "lbmh_set_speed_bound serves 1D and 2D lattices");
  for (int j = 0; j < h->dim; j++)
    if (!(abar[j] >= 0.0)) return fail(h, LBMH_ERR_INVALID_ARG, "abar must be non-negative");
  union {
    double d;
    unsigned long long u;
  } b0, b1;
  b0.d = abar[0];
  b1.d = h->dim == 2 ? abar[1] : 0.0;
  k_set_bound<<<1, 1, 0, h->stream>>>(h->ctl, current_slot(h), b0.u, b1.u);
  CK(h, cudaGetLastError());
  return LBMH_OK;
}

}  // extern "C"

namespace {

// the speed bound the step reading `slot` uses (bit patterns of non-negative
// doubles, as the side outputs store them)
__global__ void k_set_bound(Ctl* ctl, int slot, unsigned long long b0, unsigned long long b1) {
  ctl->amax[slot][0] = b0;
  ctl->amax[slot][1] = b1;
}

// three rows of every plane of the current state <-> a contiguous block
int halo_copy(lbmh_handle* h, int row, void* dev_rows, bool to_rows) {
  const long long n = 3ll * h->P.pitch * h->Q * h->m;
  if (h->prec == LBMH_FP32)
    k_halo_rows<float><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, h->Q * h->m, (float* const*)h->dbuf, h->ctl,
                                                                current_slot(h), row, (float*)dev_rows, to_rows);
  else
    k_halo_rows<double><<<blocks_for(n), kBlock, 0, h->stream>>>(h->P, h->Q * h->m, (double* const*)h->dbuf, h->ctl,
                                                                 current_slot(h), row, (double*)dev_rows, to_rows);
  CK(h, cudaGetLastError());
  return LBMH_OK;
}

size_t halo_bytes(const lbmh_handle* h) { return (size_t)3 * h->P.pitch * h->Q * h->m * h->elem; }

}  // namespace

extern "C" {

int lbmh_halo_get(lbmh_handle* h, int side, void* rows, int on_device) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!rows || (side != 0 && side != 1)) return fail(h, LBMH_ERR_INVALID_ARG, "rows is NULL or side is not 0/1");
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  if ((side == 0 ? h->halo_lo : h->halo_hi) == 0) return fail(h, LBMH_ERR_INVALID_ARG, "no neighbouring slab on that side");
  h->err.clear();
  const size_t bytes = halo_bytes(h);
  const int row = side == 0 ? h->P.ywin0 : h->P.ywin1 - 3;
  if (on_device) return halo_copy(h, row, rows, true);
  int rc = ensure_utmp(h, bytes);
  if (rc) return rc;
  rc = halo_copy(h, row, h->Utmp, true);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(rows, h->Utmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  return sync(h);
}

int lbmh_halo_set(lbmh_handle* h, int side, const void* rows, int on_device) {
  if (!h) return LBMH_ERR_INVALID_ARG;
  if (!rows || (side != 0 && side != 1)) return fail(h, LBMH_ERR_INVALID_ARG, "rows is NULL or side is not 0/1");
  if (!h->has_state) return fail(h, LBMH_ERR_INVALID_ARG, "no state");
  if ((side == 0 ? h->halo_lo : h->halo_hi) == 0) return fail(h, LBMH_ERR_INVALID_ARG, "no neighbouring slab on that side");
  h->err.clear();
  const size_t bytes = halo_bytes(h);
  const int row = side == 0 ? h->P.ywin0 - 3 : h->P.ywin1;
  if (on_device) return halo_copy(h, row, const_cast<void*>(rows), false);
  int rc = ensure_utmp(h, bytes);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(h->Utmp, rows, bytes, cudaMemcpyHostToDevice, h->stream));
  rc = halo_copy(h, row, h->Utmp, false);
  if (rc) return rc;
  return sync(h);  // the staging buffer is reused by the next host transfer
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single step
//
// For callers that must not allocate device memory: code running where
// cudaMalloc is unavailable or forbidden (inside a host callback or a
// memory-pool-only runtime, under an allocator that must stay frozen after
// start-up, or a real-time loop that cannot afford an allocation's implicit
// synchronisation).  The step runs the unfused kernels with their scratch
// (ghost-extended U, nu, omega, the control block and the per-block sums)
// placed in one file-scope device array of kStaticScratchBytes that every
// GPU loading this library holds until the process exits.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices];  // device address of g_static_scratch, per device

// control block and distribution-pointer pair of the allocation-free step
__global__ void k_static_begin(Ctl* ctl, void** bufs, void* f_in, void* f_out) {
  unsigned char* c = (unsigned char*)ctl;
  for (size_t i = 0; i < sizeof(Ctl); i++) c[i] = 0;
  bufs[0] = f_in;
  bufs[1] = f_out;
}

template <int SYS, int D>
void static_step_launch(const DevParams& P, const ExtGeom& G, Ctl* ctl, double* const* bufs, double* partials,
                        double* Ue, double* nue, double* ome, cudaStream_t stream) {
  long long nn = (long long)P.nx * P.ny;
  long long next = (long long)G.ex * G.ey;
  unsigned nb = blocks_for(next), nbn = blocks_for(nn);
  k_speed_of_f<SYS, D, double><<<nbn, kBlock, 0, stream>>>(P, bufs, ctl);
  k_moments_ext<SYS, D, double><<<nb, kBlock, 0, stream>>>(P, bufs, ctl, 0, G, Ue);
  k_indicator<SYS, D, double><<<nb, kBlock, 0, stream>>>(P, ctl, 0, G, Ue, nue);
  k_omega<D, double><<<nb, kBlock, 0, stream>>>(P, ctl, 0, G, nue, ome);
  k_collide_stream<SYS, D, double><<<nbn, kBlock, 0, stream>>>(P, bufs, ctl, 0, G, Ue, ome, partials);
}

}  // namespace

extern "C" int lbmh_step_static(const lbmh_problem* p, const double* f_in, double* f_out, double* dt_out,
                                uint32_t* status_out) {
  std::string why;
  int rc = validate(p, why);
  if (rc) return fail(nullptr, rc, why);
  if (p->precision != LBMH_FP64) return fail(nullptr, LBMH_ERR_UNSUPPORTED, "lbmh_step_static runs in FP64 only");
  if (needs_fused(p)) return fail(nullptr, LBMH_ERR_UNSUPPORTED, "lbmh_step_static has no reflecting/inflow sides or sponge");
  if (p->dim == 3) return fail(nullptr, LBMH_ERR_UNSUPPORTED, "lbmh_step_static serves 1D and 2D lattices");
  if (!f_in || !f_out || f_in == f_out) return fail(nullptr, LBMH_ERR_INVALID_ARG, "f_in and f_out must be distinct device arrays");
  const int m = nfields(p->system, p->dim), Q = 2 * p->dim + 1;
  const DevParams P = make_devparams(p, p->nx);  // the caller's arrays are unpadded [Q][m][ny][nx]
  ExtGeom G;
  G.ex = P.nx + 2 * GH;
  G.gy = p->dim == 2 ? GH : 0;
  G.ey = p->dim == 2 ? P.ny + 2 * GH : 1;

  // scratch layout: control block | pointer pair | per-block sums | U_ext | nu_ext | omega_ext
  const long long nn = (long long)P.nx * P.ny, next = (long long)G.ex * G.ey;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t off_bufs = up(sizeof(Ctl));
  const size_t off_part = off_bufs + 256;
  const size_t off_U = off_part + up((size_t)blocks_for(nn) * m * sizeof(double));
  const size_t off_nu = off_U + up((size_t)next * m * sizeof(double));
  const size_t off_om = off_nu + up((size_t)next * sizeof(double));
  const size_t need = off_om + up((size_t)next * sizeof(double));
  if (need > kStaticScratchBytes)
    return fail(nullptr, LBMH_ERR_INVALID_ARG,
                "grid too large for the static scratch: needs " + std::to_string(need) + " bytes, the limit is " +
                    std::to_string(kStaticScratchBytes) + " bytes (16 MiB)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, LBMH_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, LBMH_ERR_UNSUPPORTED, "device index beyond the static table");
  cudaStream_t stream = (cudaStream_t)p->cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return fail(nullptr, LBMH_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  void* base = nullptr;
  {
    // Outside a capture the array's device address is looked up on every call
    // (a context torn down and recreated may place the module elsewhere); under
    // a capture, where the lookup may not run, the address cached by an earlier
    // call on this device is used.
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_static_scratch);
      if (e != cudaSuccess)
        return fail(nullptr, LBMH_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_static_addr[dev] = a;
    } else if (!g_static_addr[dev]) {
      return fail(nullptr, LBMH_ERR_INVALID_ARG,
                  "lbmh_step_static under stream capture needs an earlier call on this device outside a capture");
    }
    base = g_static_addr[dev];
  }
  unsigned char* b = (unsigned char*)base;
  Ctl* ctl = (Ctl*)b;
  double** bufs = (double**)(b + off_bufs);
  double* partials = (double*)(b + off_part);
  double* Ue = (double*)(b + off_U);
  double* nue = (double*)(b + off_nu);
  double* ome = (double*)(b + off_om);

  // the kernels address node (i, j) of plane q at q*plane + j*pitch + i + XPAD;
  // shifting the base pointers by -XPAD maps that onto the unpadded arrays
  k_static_begin<<<1, 1, 0, stream>>>(ctl, (void**)bufs, (void*)(f_in - XPAD), (void*)(f_out - XPAD));
  switch (p->system * 2 + (p->dim - 1)) {
    case SYS_ADV * 2 + 0: static_step_launch<SYS_ADV, 1>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_ADV * 2 + 1: static_step_launch<SYS_ADV, 2>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_EULER * 2 + 0: static_step_launch<SYS_EULER, 1>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_EULER * 2 + 1: static_step_launch<SYS_EULER, 2>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_SWE * 2 + 0: static_step_launch<SYS_SWE, 1>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_SWE * 2 + 1: static_step_launch<SYS_SWE, 2>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_REACT * 2 + 0: static_step_launch<SYS_REACT, 1>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    case SYS_REACT * 2 + 1: static_step_launch<SYS_REACT, 2>(P, G, ctl, bufs, partials, Ue, nue, ome, stream); break;
    default: return fail(nullptr, LBMH_ERR_INVALID_ARG, "unknown system");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, LBMH_ERR_CUDA, std::string("static step launch: ") + cudaGetErrorString(e));
  if (dt_out || status_out) {
    Ctl c;
    e = cudaMemcpyAsync(&c, ctl, sizeof c, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(nullptr, LBMH_ERR_CUDA, std::string("static step readback: ") + cudaGetErrorString(e));
    if (dt_out) *dt_out = c.last_dt;
    if (status_out) *status_out = c.status;
    if (c.status & ST_BOUNDS) return fail(nullptr, LBMH_ERR_BOUNDS, "an index left its array (bounds-checked build)");
    if (c.status & ST_NONPHYSICAL) return fail(nullptr, LBMH_ERR_NONPHYSICAL, "the step produced a non-physical state");
  }
  (void)Q;
  return LBMH_OK;
}
