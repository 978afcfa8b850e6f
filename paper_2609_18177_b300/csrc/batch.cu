// Batched lattices: many 2D grids of one system and precision, of uneven
// sizes, advanced together by one persistent launch per step.
//
// Device side: an instance table (problem constants, TMA descriptors of both
// distribution buffers, control block) and a work list of strip segments
// (instance, strip, band of rows) that the resident CTAs take one at a time
// from a shared counter, so the load balances whatever the mix of grid sizes,
// and the segments of lattices that have already finished cost the CTA that
// takes them only a read of their control block.  Each instance keeps its
// own time step (Eq. 2.21 from its own speed bound), time and step count in its
// control block, and stops by itself once it reached its step target or end
// time.  Host side: admission into a fixed device arena by footprint (first-fit
// free list), work-list rebuilds, replay of a captured 3-step CUDA graph, and
// an autotuner that times the kernel variants (ring depth, segment length) on
// the live batch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/lbmh.h"
#include "common.cuh"
#include "fused.cuh"
#include "host_util.h"
#include "physics.cuh"
#include "state.cuh"

namespace lbmh {

// One lattice of a batch, as the kernel sees it (global memory, 128-byte
// aligned so the tensor maps keep their 64-byte alignment).
struct alignas(128) BatchInst {
  CUtensorMap tml[2];  // loads: padded rows of buffer b
  CUtensorMap tms[2];  // stores: interior columns of buffer b
  DevParams P;
  void* buf[2];
  Ctl* ctl;
  int strips, nxs;
};

// A strip segment: rows [yb, ye) of strip `strip` of instance `inst`.  The
// first segment of an instance in the list (owner) advances its control block.
struct BatchSeg {
  int inst, strip, yb, ye, owner, pad[3];
};

// queue[0]: next segment to take; queue[1]: CTAs done; queue[2]: segments in
// the list (written by the host with the list, so a captured graph stays valid
// when lattices come and go).  The last CTA to finish resets the two counters
// for the next launch (every CTA has stopped taking segments by then), so the
// launches of a captured graph need no host work in between.
// resident CTAs per SM the register allocation must leave room for: four for
// the FP32 advection, Euler and shallow-water steps (128 registers, what the
// step needs without spilling), two for FP32 reactive Euler (its ring and
// staged row allow two), whatever fits in FP64
template <int SYS, class R>
constexpr int batch_min_blocks() { return sizeof(R) == 8 ? 1 : (SYS == SYS_REACT ? 2 : 4); }

template <int SYS, class R, int PREF>
__global__ void __launch_bounds__(FT, batch_min_blocks<SYS, R>()) k_batch2d(const BatchInst* insts, const BatchSeg* segs, int* queue, int slot,
                                                double* seg_sums) {
  constexpr int M = Fields<SYS, 2>::M;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_abort;
  __shared__ int s_seg;
  // step coefficients of the current segment's lattice: FP64 arithmetic done
  // once by thread 0, not by every thread of every segment
  __shared__ StepCoef s_cf;
  __shared__ Coef2D<R> s_cc;
  const int t = threadIdx.x;
  Pipe2D pp;
  pipe2d_init<SYS, R, PREF, 1>(pp, smem_raw, &s_abort);
  const int nsegs = queue[2];
  for (;;) {
    // (every thread read the previous s_seg before the s_cf barrier below)
    if (t == 0) s_seg = atomicAdd(&queue[0], 1);
    __syncthreads();
    const int i = s_seg;
    if (i >= nsegs) break;
    const BatchSeg sg = segs[i];
    const BatchInst& I = insts[sg.inst];
    const DevParams P = I.P;
    Ctl* ctl = I.ctl;
    if (t == 0) {
      s_cf = step_coef<2>(P, ctl, slot);
      s_cc = make_coef2d<R>(s_cf, P);
    }
    __syncthreads();  // (the previous segment's readers passed the segment barrier above)
    const StepCoef cf = s_cf;
    if (!cf.active) {  // a finished lattice: only its owner segment moves the control block on
      if (sg.owner && t == 0) advance_ctl<2>(ctl, slot, cf);
      continue;
    }
    R sp0 = R(0), sp1 = R(0);
    Acc<R> acc[M];
#pragma unroll
    for (int c = 0; c < M; c++) acc[c].init();
    unsigned st = 0u;
    if (!pp.aborted) {
      const int par = ctl->parity[slot];
      const CUtensorMap* tml = &I.tml[par];
      const CUtensorMap* tms = &I.tms[par ^ 1];
      if (t == 0) {  // the descriptors live in global memory
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tml) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tms) : "memory");
      }
      const Phys<R> K = make_phys<R>(P);
      const Coef2D<R> cc = s_cc;
      run_segment2d<SYS, R, PREF, 1>(pp, tml, tms, (R*)I.buf[par ^ 1], P, K, cc, sg.strip, sg.yb, sg.ye, I.nxs, sp0,
                                     sp1, acc, st, &ctl->status);
      if (pp.aborted) st |= ST_TIMEOUT;
    } else {
      st |= ST_TIMEOUT;  // an earlier wait of this CTA gave up: this segment's rows were not written
    }
    // this segment's side outputs: speed bound of its instance, FP64 sums
    fused_side_outputs_to<M, R>(sp0, sp1, acc, ctl, (slot + 1) % 3, seg_sums + (long long)i * M, st);
    if (sg.owner && t == 0) advance_ctl<2>(ctl, slot, cf);
  }
  pipe2d_drain<SYS, R, PREF, 1>(pp);
  if (t == 0) {
    __threadfence();
    if (atomicAdd(&queue[1], 1) == (int)gridDim.x - 1) {
      queue[0] = 0;
      queue[1] = 0;
    }
  }
}

// U = sum_k f_k of one batch instance into FP64 [m][ny][nx]
template <int M, class R>
__global__ void k_batch_moments(DevParams P, const R* f, double* U, Ctl* ctl) {
  long long nn = (long long)P.nx * P.ny;
  long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int j = (int)(node / P.nx), i = (int)(node % P.nx);
  long long off = cell(P, i, j);
#pragma unroll
  for (int c = 0; c < M; c++) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < 5; k++) s += f[chk((long long)(k * M + c) * P.plane + off, 5ll * M * P.plane, &ctl->status)];
    U[c * nn + node] = (double)s;
  }
}

// move the initial state of a control block from slot 0 to slot s
__global__ void k_ctl_to_slot(Ctl* ctl, int s) {
  if (s == 0) return;
  ctl->amax[s][0] = ctl->amax[0][0];
  ctl->amax[s][1] = ctl->amax[0][1];
  ctl->t[s] = ctl->t[0];
  ctl->nsteps[s] = ctl->nsteps[0];
  ctl->parity[s] = ctl->parity[0];
  ctl->amax[0][0] = ctl->amax[0][1] = 0ull;
  ctl->t[0] = 0.0;
  ctl->nsteps[0] = 0;
  ctl->parity[0] = 0;
}

}  // namespace lbmh

using namespace lbmh;

namespace {

constexpr int kPrefVariants[2] = {1, 2};
constexpr int kBands[4] = {64, 128, 256, 512};  // rows per segment

struct InstHost {
  bool used = false;
  lbmh_problem prob;
  DevParams P;
  size_t off[2] = {0, 0};  // arena offsets of the two buffers
  size_t bytes = 0;        // per buffer
  int strips = 0;
};

struct Block {
  size_t off, size;
};

}  // namespace

struct lbmh_batch {
  int sys, prec, m, Q;
  size_t elem;
  cudaStream_t stream;
  int max_inst;
  size_t capacity;
  unsigned char* arena;
  std::vector<Block> free_list;  // sorted by offset, coalesced
  size_t used_bytes;
  std::vector<InstHost> inst;
  std::vector<BatchInst> h_insts;
  BatchInst* d_insts;
  Ctl* d_ctl;
  BatchSeg* d_segs;
  int seg_cap;
  int* d_queue;  // segment counter and finished-CTA counter of the running launch
  double* d_sums;
  double* staging;
  size_t staging_bytes;
  int nsegs;
  std::vector<BatchSeg> h_segs;
  std::vector<int> seg_inst_first;
  long long launched;
  int grid[2];     // resident CTAs per PREF variant
  int variant;     // index into kPrefVariants
  int band;        // index into kBands
  bool tuned;
  cudaStream_t cap_stream;  // private stream the step graph is captured on
  cudaGraphExec_t graph;
  bool graph_ok;
  int graph_variant;
  std::string err;
};

namespace {

std::string g_batch_error;

int bfail(lbmh_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg; else g_batch_error = msg;
  return code;
}

#define BCK(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return bfail(b, LBMH_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

bool arena_alloc(lbmh_batch* b, size_t bytes, size_t* off) {
  bytes = (bytes + 255) / 256 * 256;
  for (size_t i = 0; i < b->free_list.size(); i++) {
    Block& f = b->free_list[i];
    if (f.size >= bytes) {
      *off = f.off;
      f.off += bytes;
      f.size -= bytes;
      if (f.size == 0) b->free_list.erase(b->free_list.begin() + i);
      b->used_bytes += bytes;
      return true;
    }
  }
  return false;
}

void arena_free(lbmh_batch* b, size_t off, size_t bytes) {
  bytes = (bytes + 255) / 256 * 256;
  b->used_bytes -= bytes;
  auto it = std::lower_bound(b->free_list.begin(), b->free_list.end(), off,
                             [](const Block& x, size_t o) { return x.off < o; });
  it = b->free_list.insert(it, Block{off, bytes});
  size_t i = it - b->free_list.begin();
  if (i + 1 < b->free_list.size() && b->free_list[i].off + b->free_list[i].size == b->free_list[i + 1].off) {
    b->free_list[i].size += b->free_list[i + 1].size;
    b->free_list.erase(b->free_list.begin() + i + 1);
  }
  if (i > 0 && b->free_list[i - 1].off + b->free_list[i - 1].size == b->free_list[i].off) {
    b->free_list[i - 1].size += b->free_list[i].size;
    b->free_list.erase(b->free_list.begin() + i);
  }
}

template <int SYS, class R, int PREF>
void* batch_kernel_ptr() {
  return (void*)k_batch2d<SYS, R, PREF>;
}

template <class R>
size_t batch_smem(int sys, int pref) {
  auto f = [&](auto tag) -> size_t {
    constexpr int S = decltype(tag)::value;
    return pref == 1 ? Smem2D<Fields<S, 2>::M, R, 1, 1>::total : Smem2D<Fields<S, 2>::M, R, 2, 1>::total;
  };
  switch (sys) {
    case SYS_ADV: return f(std::integral_constant<int, SYS_ADV>());
    case SYS_EULER: return f(std::integral_constant<int, SYS_EULER>());
    case SYS_SWE: return f(std::integral_constant<int, SYS_SWE>());
    default: return f(std::integral_constant<int, SYS_REACT>());
  }
}

template <class R>
void* batch_kernel(int sys, int pref) {
#define BK(S) \
  case S: return pref == 1 ? batch_kernel_ptr<S, R, 1>() : batch_kernel_ptr<S, R, 2>();
  switch (sys) {
    BK(SYS_ADV)
    BK(SYS_EULER)
    BK(SYS_SWE)
    BK(SYS_REACT)
  }
#undef BK
  return nullptr;
}

void* kernel_of(const lbmh_batch* b, int variant) {
  int pref = kPrefVariants[variant];
  return b->prec == LBMH_FP32 ? batch_kernel<float>(b->sys, pref) : batch_kernel<double>(b->sys, pref);
}

size_t smem_of(const lbmh_batch* b, int variant) {
  int pref = kPrefVariants[variant];
  return b->prec == LBMH_FP32 ? batch_smem<float>(b->sys, pref) : batch_smem<double>(b->sys, pref);
}

// work list: bands of rows of every strip of every live instance, larger
// lattices first (their segments are taken first, the small ones fill the
// tail of the step), band-major within a lattice so that neighbouring strips
// of a band run side by side and share their halo sectors in L2
int rebuild_worklist(lbmh_batch* b) {
  const int band = kBands[b->band];
  std::vector<int> order;
  for (int i = 0; i < b->max_inst; i++)
    if (b->inst[i].used) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return (long long)b->inst[a].strips * b->inst[a].P.ny > (long long)b->inst[c].strips * b->inst[c].P.ny;
  });
  std::vector<BatchSeg> segs;
  for (int i : order) {
    const InstHost& ih = b->inst[i];
    const int ny = ih.P.ny;
    for (int y0 = 0; y0 < ny; y0 += band)
      for (int s = 0; s < ih.strips; s++) segs.push_back(BatchSeg{i, s, y0, std::min(ny, y0 + band), 0, {0, 0, 0}});
  }
  std::vector<char> seen(b->max_inst, 0);
  for (BatchSeg& sg : segs)
    if (!seen[sg.inst]) {
      sg.owner = 1;
      seen[sg.inst] = 1;
    }
  if ((int)segs.size() > b->seg_cap) {
    cudaStreamSynchronize(b->stream);
    cudaFree(b->d_segs);
    cudaFree(b->d_sums);
    b->seg_cap = (int)segs.size() * 2;
    if (cudaMalloc(&b->d_segs, sizeof(BatchSeg) * b->seg_cap) != cudaSuccess ||
        cudaMalloc(&b->d_sums, sizeof(double) * b->m * b->seg_cap) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, LBMH_ERR_OOM, "work list allocation failed");
    }
    b->graph_ok = false;  // the captured launches hold the old pointers
  }
  b->h_segs = segs;
  b->nsegs = (int)segs.size();
  if (!segs.empty())
    BCK(b, cudaMemcpyAsync(b->d_segs, segs.data(), sizeof(BatchSeg) * segs.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_queue + 2, &b->nsegs, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  // the host vectors must outlive the asynchronous copies
  BCK(b, cudaStreamSynchronize(b->stream));
  return LBMH_OK;
}

int launch_one(lbmh_batch* b, int variant, cudaStream_t stream) {
  const int G = b->grid[variant];
  int slot = (int)(b->launched % 3);
  void* args[] = {(void*)&b->d_insts, (void*)&b->d_segs, (void*)&b->d_queue, (void*)&slot, (void*)&b->d_sums};
  BCK(b, cudaLaunchKernel(kernel_of(b, variant), dim3(G), dim3(FT), args, smem_of(b, variant), stream));
  b->launched++;
  return LBMH_OK;
}

int launch_one(lbmh_batch* b, int variant) { return launch_one(b, variant, b->stream); }

// Three steps (slots 0, 1, 2) captured on the batch's private stream; the
// caller's stream may be the legacy default stream, which cannot be captured.
int capture_graph(lbmh_batch* b) {
  if (b->graph_ok) {
    cudaGraphExecDestroy(b->graph);
    b->graph_ok = false;
  }
  cudaGraph_t g = nullptr;
  long long saved = b->launched;
  b->launched = 0;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? LBMH_OK : bfail(b, LBMH_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  for (int i = 0; i < 3 && rc == LBMH_OK; i++) rc = launch_one(b, b->variant, b->cap_stream);
  if (e == cudaSuccess) {
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc == LBMH_OK && e2 != cudaSuccess)
      rc = bfail(b, LBMH_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e2));
  }
  b->launched = saved;
  if (rc == LBMH_OK) {
    e = cudaGraphInstantiate(&b->graph, g, 0);
    if (e != cudaSuccess) rc = bfail(b, LBMH_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  if (g) cudaGraphDestroy(g);
  if (rc != LBMH_OK) {
    cudaGetLastError();  // leave no sticky error behind
    return rc;
  }
  b->graph_ok = true;
  b->graph_variant = b->variant;
  return LBMH_OK;
}

void free_batch(lbmh_batch* b) {
  if (!b) return;
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->arena);
  cudaFree(b->d_insts);
  cudaFree(b->d_ctl);
  cudaFree(b->d_segs);
  cudaFree(b->d_queue);
  cudaFree(b->d_sums);
  cudaFree(b->staging);
  delete b;
}

int ensure_staging(lbmh_batch* b, size_t bytes) {
  if (b->staging_bytes >= bytes) return LBMH_OK;
  cudaStreamSynchronize(b->stream);
  cudaFree(b->staging);
  b->staging = nullptr;
  b->staging_bytes = 0;
  if (cudaMalloc((void**)&b->staging, bytes) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, LBMH_ERR_OOM, "staging allocation failed");
  }
  b->staging_bytes = bytes;
  return LBMH_OK;
}

template <int SYS, class R>
int init_instance(lbmh_batch* b, int i, const double* U0dev) {
  InstHost& ih = b->inst[i];
  const DevParams& P = ih.P;
  long long nn = (long long)P.nx * P.ny;
  Ctl* ctl = b->d_ctl + i;
  R* f0 = (R*)(b->arena + ih.off[0]);
  BCK(b, cudaMemsetAsync(ctl, 0, sizeof(Ctl), b->stream));
  k_init_speed<SYS, 2><<<reduce_blocks_for(nn), kBlock, 0, b->stream>>>(P, U0dev, ctl);
  k_init_eq<SYS, 2, R><<<reduce_blocks_for(nn), kBlock, 0, b->stream>>>(P, U0dev, f0, ctl);
  long long npad = (long long)P.ny * b->Q * b->m * 2 * NGHOST;
  k_fill_pads<R><<<blocks_for(npad), kBlock, 0, b->stream>>>(P, b->Q * b->m, f0, ctl);
  k_ctl_to_slot<<<1, 1, 0, b->stream>>>(ctl, (int)(b->launched % 3));
  BCK(b, cudaGetLastError());
  return LBMH_OK;
}

int init_dispatch(lbmh_batch* b, int i, const double* U0dev) {
#define ID(S) \
  case S: return b->prec == LBMH_FP32 ? init_instance<S, float>(b, i, U0dev) : init_instance<S, double>(b, i, U0dev);
  switch (b->sys) {
    ID(SYS_ADV)
    ID(SYS_EULER)
    ID(SYS_SWE)
    ID(SYS_REACT)
  }
#undef ID
  return bfail(b, LBMH_ERR_INVALID_ARG, "unknown system");
}

template <class R>
int moments_of(lbmh_batch* b, int i, int par, double* Udev) {
  InstHost& ih = b->inst[i];
  long long nn = (long long)ih.P.nx * ih.P.ny;
  const R* f = (const R*)(b->arena + ih.off[par]);
  switch (b->m) {
    case 1: k_batch_moments<1, R><<<blocks_for(nn), kBlock, 0, b->stream>>>(ih.P, f, Udev, b->d_ctl + i); break;
    case 3: k_batch_moments<3, R><<<blocks_for(nn), kBlock, 0, b->stream>>>(ih.P, f, Udev, b->d_ctl + i); break;
    case 4: k_batch_moments<4, R><<<blocks_for(nn), kBlock, 0, b->stream>>>(ih.P, f, Udev, b->d_ctl + i); break;
    case 5: k_batch_moments<5, R><<<blocks_for(nn), kBlock, 0, b->stream>>>(ih.P, f, Udev, b->d_ctl + i); break;
    default: return bfail(b, LBMH_ERR_INVALID_ARG, "unsupported field count");
  }
  BCK(b, cudaGetLastError());
  return LBMH_OK;
}

}  // namespace

extern "C" {

int lbmh_batch_create(int system, int precision, int64_t capacity_bytes, int max_instances, void* cuda_stream,
                      lbmh_batch** out) {
  if (!out) return bfail(nullptr, LBMH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (system < 0 || system > 3) return bfail(nullptr, LBMH_ERR_INVALID_ARG, "unknown or unsupported system");
  if (precision != LBMH_FP32 && precision != LBMH_FP64) return bfail(nullptr, LBMH_ERR_INVALID_ARG, "bad precision");
  if (capacity_bytes <= 0 || max_instances < 1 || max_instances > 65536)
    return bfail(nullptr, LBMH_ERR_INVALID_ARG, "capacity and instance count must be positive");
  lbmh_batch* b = new lbmh_batch();
  b->sys = system;
  b->prec = precision;
  b->m = nfields(system, 2);
  b->Q = 5;
  b->elem = precision == LBMH_FP32 ? 4 : 8;
  b->stream = (cudaStream_t)cuda_stream;
  b->max_inst = max_instances;
  b->capacity = (size_t)capacity_bytes;
  b->arena = nullptr;
  b->used_bytes = 0;
  b->inst.assign(max_instances, InstHost());
  b->h_insts.assign(max_instances, BatchInst());
  b->d_insts = nullptr;
  b->d_ctl = nullptr;
  b->d_segs = nullptr;
  b->d_queue = nullptr;
  b->d_sums = nullptr;
  b->staging = nullptr;
  b->staging_bytes = 0;
  b->nsegs = 0;
  b->seg_cap = 4096;
  b->launched = 0;
  b->variant = 1;  // PREF 2
  b->band = 2;  // 256 rows
  b->tuned = false;
  b->graph_ok = false;
  b->graph_variant = -1;
  b->cap_stream = nullptr;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return bfail(nullptr, LBMH_ERR_CUDA, "stream creation failed");
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int v = 0; v < 2; v++) {
    void* k = kernel_of(b, v);
    size_t smem = smem_of(b, v);
    int per_sm = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, FT, smem) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      free_batch(b);
      return bfail(nullptr, LBMH_ERR_CUDA, "batch kernel does not fit on this device");
    }
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    b->grid[v] = per_sm * sms;
  }
  if (cudaMalloc((void**)&b->arena, b->capacity) != cudaSuccess ||
      cudaMalloc((void**)&b->d_insts, sizeof(BatchInst) * max_instances) != cudaSuccess ||
      cudaMalloc((void**)&b->d_ctl, sizeof(Ctl) * max_instances) != cudaSuccess ||
      cudaMalloc((void**)&b->d_segs, sizeof(BatchSeg) * b->seg_cap) != cudaSuccess ||
      cudaMalloc((void**)&b->d_queue, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc((void**)&b->d_sums, sizeof(double) * b->m * b->seg_cap) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return bfail(nullptr, LBMH_ERR_OOM, "batch device allocation failed");
  }
  cudaMemset(b->d_ctl, 0, sizeof(Ctl) * max_instances);
  cudaMemset(b->d_queue, 0, sizeof(int) * 4);
  b->free_list.push_back(Block{0, b->capacity});
  *out = b;
  return LBMH_OK;
}

int lbmh_batch_destroy(lbmh_batch* b) {
  if (!b) return LBMH_OK;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  return LBMH_OK;
}

const char* lbmh_batch_last_error(const lbmh_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

int64_t lbmh_batch_footprint(const lbmh_problem* p) {
  if (!p || p->dim != 2 || p->nx < 1 || p->ny < 1) return -1;
  size_t elem = p->precision == LBMH_FP32 ? 4 : 8;
  int m = nfields(p->system, 2);
  if (m < 1) return -1;
  size_t per = (size_t)5 * m * p->ny * padded_pitch(p->nx, elem) * elem;
  return (int64_t)(2 * ((per + 255) / 256 * 256));
}

int lbmh_batch_add(lbmh_batch* b, const lbmh_problem* p, const double* U0, int on_device, int64_t max_steps, double T,
                   int* slot_out) {
  if (!b || !p || !U0 || !slot_out) return LBMH_ERR_INVALID_ARG;
  b->err.clear();
  std::string why;
  int rc = validate(p, why);
  if (rc) return bfail(b, rc, why);
  if (p->system != b->sys || p->dim != 2 || p->precision != b->prec)
    return bfail(b, LBMH_ERR_INVALID_ARG, "problem does not match the batch (system, 2D, precision)");
  int i = -1;
  for (int k = 0; k < b->max_inst; k++)
    if (!b->inst[k].used) {
      i = k;
      break;
    }
  if (i < 0) return bfail(b, LBMH_ERR_OOM, "no free instance slot");
  InstHost ih;
  ih.used = true;
  ih.prob = *p;
  ih.P = make_devparams(p, padded_pitch(p->nx, b->elem));
  apply_wait_hook(ih.P);
  ih.P.max_steps = max_steps > 0 ? max_steps : 0;
  ih.P.T = T > 0.0 ? T : 0.0;
  ih.bytes = (size_t)b->Q * b->m * ih.P.plane * b->elem;
  if (!arena_alloc(b, ih.bytes, &ih.off[0])) return bfail(b, LBMH_ERR_OOM, "batch arena full");
  if (!arena_alloc(b, ih.bytes, &ih.off[1])) {
    arena_free(b, ih.off[0], ih.bytes);
    return bfail(b, LBMH_ERR_OOM, "batch arena full");
  }
  BatchInst& bi = b->h_insts[i];
  memset(&bi, 0, sizeof bi);
  bi.P = ih.P;
  bi.buf[0] = b->arena + ih.off[0];
  bi.buf[1] = b->arena + ih.off[1];
  bi.ctl = b->d_ctl + i;
  FusedPlan fp;
  memset(&fp, 0, sizeof fp);
  int e2 = b->prec == LBMH_FP32 ? encode_maps<float>(fp, ih.P, bi.buf, b->m * 5, FT, FW)
                                 : encode_maps<double>(fp, ih.P, bi.buf, b->m * 5, FT, FW);
  if (e2) {
    arena_free(b, ih.off[0], ih.bytes);
    arena_free(b, ih.off[1], ih.bytes);
    return bfail(b, LBMH_ERR_CUDA, "tensor map encoding failed");
  }
  for (int k = 0; k < 2; k++) {
    bi.tml[k] = fp.tm[k];
    bi.tms[k] = fp.tms[k];
  }
  bi.strips = fp.strips;
  bi.nxs = fp.nxs;
  ih.strips = fp.strips;
  b->inst[i] = ih;
  BCK(b, cudaMemcpyAsync(b->d_insts + i, &bi, sizeof bi, cudaMemcpyHostToDevice, b->stream));
  long long nn = (long long)ih.P.nx * ih.P.ny;
  const double* src = U0;
  if (!on_device) {
    rc = ensure_staging(b, (size_t)nn * b->m * sizeof(double));
    if (rc) return rc;
    BCK(b, cudaMemcpyAsync(b->staging, U0, (size_t)nn * b->m * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    src = b->staging;
  }
  rc = init_dispatch(b, i, src);
  if (rc) return rc;
  rc = rebuild_worklist(b);  // synchronises: the staging and the descriptor copies are done
  if (rc) return rc;
  *slot_out = i;
  return LBMH_OK;
}

int lbmh_batch_remove(lbmh_batch* b, int slot) {
  if (!b || slot < 0 || slot >= b->max_inst || !b->inst[slot].used) return LBMH_ERR_INVALID_ARG;
  BCK(b, cudaStreamSynchronize(b->stream));
  InstHost& ih = b->inst[slot];
  arena_free(b, ih.off[0], ih.bytes);
  arena_free(b, ih.off[1], ih.bytes);
  ih.used = false;
  return rebuild_worklist(b);
}

int lbmh_batch_step(lbmh_batch* b, int64_t n) {
  if (!b || n < 0) return LBMH_ERR_INVALID_ARG;
  b->err.clear();
  if (b->nsegs == 0) return LBMH_OK;
  int64_t done = 0;
  while (done < n) {
    if (b->launched % 3 == 0 && n - done >= 3) {
      if (!b->graph_ok || b->graph_variant != b->variant) {
        int rc = capture_graph(b);
        if (rc) return rc;
      }
      BCK(b, cudaGraphLaunch(b->graph, b->stream));
      b->launched += 3;
      done += 3;
    } else {
      int rc = launch_one(b, b->variant);
      if (rc) return rc;
      done++;
    }
  }
  return LBMH_OK;
}

int lbmh_batch_autotune(lbmh_batch* b, int steps_per_candidate, double* best_ms) {
  if (!b || steps_per_candidate < 1) return LBMH_ERR_INVALID_ARG;
  if (b->nsegs == 0) return LBMH_OK;
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = b->variant, best_b = b->band;
  for (int v = 0; v < 2; v++)
    for (int bi = 0; bi < 4; bi++) {
      b->variant = v;
      b->band = bi;
      int rc = rebuild_worklist(b);
      if (rc) return rc;
      rc = launch_one(b, v);  // warm-up: one real step
      if (rc) return rc;
      BCK(b, cudaEventRecord(e0, b->stream));
      for (int s = 0; s < steps_per_candidate; s++) {
        rc = launch_one(b, v);
        if (rc) return rc;
      }
      BCK(b, cudaEventRecord(e1, b->stream));
      BCK(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= steps_per_candidate;
      if (ms < best) {
        best = ms;
        best_v = v;
        best_b = bi;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = best_v;
  b->band = best_b;
  b->tuned = true;
  if (best_ms) *best_ms = best;
  return rebuild_worklist(b);
}

int lbmh_batch_poll(lbmh_batch* b, int* done, double* t, int64_t* steps, uint32_t* status) {
  if (!b) return LBMH_ERR_INVALID_ARG;
  std::vector<Ctl> c(b->max_inst);
  BCK(b, cudaMemcpyAsync(c.data(), b->d_ctl, sizeof(Ctl) * b->max_inst, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  int slot = (int)(b->launched % 3);
  for (int i = 0; i < b->max_inst; i++) {
    const InstHost& ih = b->inst[i];
    bool used = ih.used;
    long long ns = used ? c[i].nsteps[slot] : 0;
    double ti = used ? c[i].t[slot] : 0.0;
    bool fin = used && ((ih.P.max_steps > 0 && ns >= ih.P.max_steps) || (ih.P.T > 0.0 && ti >= ih.P.T) ||
                        (c[i].status & (ST_NONPHYSICAL | ST_TIMEOUT)));
    if (done) done[i] = used ? (fin ? 1 : 0) : -1;
    if (t) t[i] = ti;
    if (steps) steps[i] = ns;
    if (status) status[i] = used ? c[i].status : 0u;
  }
  return LBMH_OK;
}

int lbmh_batch_moments(lbmh_batch* b, int slot, double* U_out, int on_device) {
  if (!b || slot < 0 || slot >= b->max_inst || !b->inst[slot].used || !U_out) return LBMH_ERR_INVALID_ARG;
  Ctl c;
  BCK(b, cudaMemcpyAsync(&c, b->d_ctl + slot, sizeof c, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  int par = c.parity[b->launched % 3];
  const InstHost& ih = b->inst[slot];
  size_t bytes = (size_t)ih.P.nx * ih.P.ny * b->m * sizeof(double);
  int rc = on_device ? LBMH_OK : ensure_staging(b, bytes);
  if (rc) return rc;
  double* dst = on_device ? U_out : b->staging;
  rc = b->prec == LBMH_FP32 ? moments_of<float>(b, slot, par, dst) : moments_of<double>(b, slot, par, dst);
  if (rc) return rc;
  if (!on_device) {
    BCK(b, cudaMemcpyAsync(U_out, b->staging, bytes, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
  }
  return LBMH_OK;
}

int lbmh_batch_info(lbmh_batch* b, int64_t* used_bytes, int64_t* capacity_bytes, int* active, int* grid,
                    int* variant) {
  if (!b) return LBMH_ERR_INVALID_ARG;
  int n = 0;
  for (const InstHost& ih : b->inst) n += ih.used;
  if (used_bytes) *used_bytes = (int64_t)b->used_bytes;
  if (capacity_bytes) *capacity_bytes = (int64_t)b->capacity;
  if (active) *active = n;
  if (grid) *grid = b->grid[b->variant];
  if (variant) *variant = kPrefVariants[b->variant] * 1000 + kBands[b->band];
  return LBMH_OK;
}

}  // extern "C"
