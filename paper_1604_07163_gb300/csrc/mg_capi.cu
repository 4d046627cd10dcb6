// C ABI of the multigrid-preconditioned CG library (declarations and
// argument conventions in include/mg.h).  Host side: level hierarchy,
// launch geometry, the V-cycle driver (Algorithm 1 applied recursively),
// the float64 PCG loop and the step entry points.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "mg.h"
#include "mg_kernels.cuh"
#include "mg_tma.cuh"
#include "mg_zvec.cuh"
#include "mg_g27.cuh"
#include "mg_krylov.cuh"

using namespace mgdev;

namespace {

struct LevelBuf {
  Geom g{};
  int N[3] = {0, 0, 0};
  double ih2[3] = {0, 0, 0};       // h_a^-2
  double* kc = nullptr;            // cell k (dense)
  void *kx = nullptr, *ky = nullptr, *kz = nullptr;          // V-cycle precision
  double *kx64 = nullptr, *ky64 = nullptr, *kz64 = nullptr;  // float64 copies
  void* dinv = nullptr;
  void* x[2] = {nullptr, nullptr};
  void *d = nullptr, *b = nullptr, *r = nullptr;
  // TMA tensor maps (2-D row views) for the staged stencil kernels
  bool tma = false;
  CUtensorMap m_full_x[2], m_full_b, m_full_dinv, m_kx, m_ky, m_kz, m_c_dinv, m_c_b, m_c_d;
  int tma_grid[3] = {0, 0, 0}, tma_kchunk = 0;
  // Galerkin (27-point) level: couplings w (13 arrays, V-cycle precision) and
  // their float64 copies, diagonal in the V-cycle precision and in float64
  bool g27 = false;
  void* w = nullptr;
  double* w64 = nullptr;
  void* dg = nullptr;
  double* dg64 = nullptr;
  double beta = 2.0;   // Chebyshev interval [alpha, beta] of the level's D^-1 A
  double alpha = 0.2;
};

std::string g_setup_error;

// Named host ranges for profilers (ncu --nvtx, Nsight Systems): setup, each
// solve, each outer iteration and each V-cycle.  The NVTX v3 header is
// self-contained; with no tool attached a range costs one check of a
// function pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// One step of a recorded solve phase of a z-slab sub-hierarchy (see the
// z-slab decomposition below): a kernel launch (with the operand whose halo
// planes it reads, if any), a memset, a reduction to finish across the slabs,
// or the hand-over of the agglomeration level to the root hierarchy.
struct Pass {
  enum Kind { LAUNCH, MEMSET, FINISH, AGGLOM } kind = LAUNCH;
  std::function<void()> fn;  // LAUNCH, MEMSET
  void* halo = nullptr;      // LAUNCH: operand whose halo planes the kernel reads (null: pointwise)
  int halo_bytes = 0;        // its element size
  Geom halo_g{};             // and its level's (local) geometry
  int nb = 0, mode = 0;      // FINISH: per-block partials and the scalar update
  int level = 0;             // AGGLOM
};

}  // namespace

struct mg_handle {
  mg_params prm{};
  cudaStream_t s = nullptr;   // internal non-blocking stream (graph capture needs one)
  cudaStream_t us = nullptr;  // caller's stream; ordered against s with events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_scal = nullptr;  // the copy of the CG scalars to the host has landed
  int nsm = 152;
  int L = 0, lb = 0;  // levels; first level of the bottom kernel
  int bot_cluster = 1;  // blocks of the bottom kernel (a cluster when > 1)
  LevelBuf lv[MG_MAX_LEVELS];
  double* Lc = nullptr;  // Cholesky factor of the coarsest operator
  double* Li = nullptr;  // L^-1 and the coarsest operator inverse when that level has at most 32 unknowns
  double* Ac = nullptr;  // the dense coarsest operator (inexact coarse solve)
  // flexible GMRES: basis V_0..V_m (float64), preconditioned Z_0..Z_{m-1}
  // (V-cycle precision), one column's dots and the coefficients y, partial sums
  double* kv = nullptr;
  void* kz = nullptr;
  double* kh = nullptr;
  double* kpart = nullptr;
  double* khost = nullptr;  // pinned mirror of kh
  int kgrid = 0;
  int nc = 0;
  double *cb = nullptr, *cx = nullptr, *cr = nullptr, *cq = nullptr, *cp = nullptr;
  double* cw = nullptr;    // float64 scratch (gradient input)
  double* dg64 = nullptr;  // float64 diagonal of the finest operator
  double* partials = nullptr;
  int pstride = 0;
  Scal* dsc = nullptr;
  Scal* hsc = nullptr;      // pinned host mirror (mapped)
  Scal* hsc_dev = nullptr;  // its device address (k_finish writes the outer iteration's scalars there)
  int* dflag = nullptr;
  std::vector<double> hist;
  std::string err;
  mg_stats st{};
  std::vector<void*> allocs;
  cudaGraphExec_t vexec = nullptr;
  int vexec_zcur = 0;
  bool rz_fused = false;         // last V-cycle fused rho = b.z (OpChebStepDot) into its final step
  bool zvec = true;              // stencil passes on the two-points-per-thread driver (k_zvec)
  int lin_grid = 0;              // largest grid of the linear (pointwise) kernels
  long long launches = 0;        // kernels launched (counted at launch sites)
  long long graph_launches = 0;  // kernels inside the captured V-cycle graph
  // opt-in kernel timing
  struct TRec {
    int cls, level;
    double pts;
    int ev;  // index of the start event; ev + 1 is the stop event
  };
  bool timing = false;
  int t_cls_mask = 0, t_lvl_mask = 0;
  bool capturing = false;
  std::vector<cudaEvent_t> evpool;
  int ev_graph_end = 0;  // events [0, ev_graph_end) belong to the captured graph
  int ev_next = 0;
  std::vector<TRec> graph_recs, pending;
  cudaEvent_t gap_ev[2][2] = {};  // host-gap timing: two alternating (end of iteration, next launch) pairs
  double* hstage[2] = {nullptr, nullptr};  // dense device nodal arrays of mg_solve_host (f, x)
  double t_ms[MG_K_NCLASS][MG_MAX_LEVELS] = {};
  long long t_n[MG_K_NCLASS][MG_MAX_LEVELS] = {};
  double t_pts[MG_K_NCLASS][MG_MAX_LEVELS] = {};
  // z-slab decomposition (mg_params.slabs > 1).  A slab sub-hierarchy records
  // its launches into rec instead of issuing them; halo_* name the operand of
  // the next recorded launch; pointwise kernels of a sub-hierarchy cover its
  // interior planes [lin_lo, lin_hi) only (its pad planes hold neighbours'
  // halo planes).
  std::vector<Pass>* rec = nullptr;
  mutable void* halo_ptr = nullptr;
  mutable int halo_bytes = 0;
  mutable Geom halo_g{};
  i64 lin_lo = 0, lin_hi = -1;
  bool sub = false;                    // a slab sub-hierarchy (stream and scalars are the parent's)
  int nslab = 1, la = 0;               // parent: slabs and agglomeration level
  int slab_first = 0;                  // parent: global index of its first (in rank mode: only) slab
  bool rank_mode = false;              // parent: holds one slab and talks to the other ranks through tr
  mg_transport tr{};
  bool tr_set = false;
  std::vector<mg_handle*> slab;        // parent: the slab sub-hierarchies
  std::vector<int> slab_z0;            // parent: first interior plane of slab s on level l at l*(nslab+1)+s
  double* slots = nullptr;             // parent: per-slab reduction slots (2 x nslab)
  std::vector<std::vector<Pass>> vrec, crec;  // parent: each slab's recorded V-cycle and CG iteration
  std::vector<void*> vz;               // parent: each slab's V-cycle output buffer
};

namespace {

// One thread-block cluster of nb blocks (a bottom kernel whose passes are
// split over nb SMs).
template <class... KArgs, class... Args>
void launch_cluster(const mg_handle* h, void (*kern)(KArgs...), int nb, dim3 block, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = block;
  cfg.stream = h->s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = h->prm.use_pdl ? 1 : 0;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = nb;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <class... KArgs, class... Args>
void launch_now(const mg_handle* h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h->s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = h->prm.use_pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Launch on the handle's stream; a slab sub-hierarchy in recording mode keeps
// the launch (with its arguments and the operand named by halo_*) for replay.
template <class... KArgs, class... Args>
void launch(const mg_handle* h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args) {
  if (h->rec) {
    Pass ps;
    ps.kind = Pass::LAUNCH;
    ps.halo = h->halo_ptr;
    ps.halo_bytes = h->halo_bytes;
    ps.halo_g = h->halo_g;
    h->halo_ptr = nullptr;
    auto tup = std::make_tuple(std::decay_t<Args>(args)...);
    ps.fn = [h, kern, grid, block, smem, tup]() {
      std::apply([&](const auto&... a) { launch_now(h, kern, grid, block, smem, a...); }, tup);
    };
    h->rec->push_back(std::move(ps));
    return;
  }
  launch_now(h, kern, grid, block, smem, std::forward<Args>(args)...);
}

using clk = std::chrono::steady_clock;
double secs(clk::time_point a) { return std::chrono::duration<double>(clk::now() - a).count(); }

mg_status fail(mg_handle* h, mg_status code, const std::string& msg) {
  if (h) h->err = msg;
  else g_setup_error = msg;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(h, MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define CKL() CK(cudaGetLastError())

int roundup(int a, int m) { return (a + m - 1) / m * m; }

// Plane split for tiles x zs blocks: the split with the best wave efficiency
// (blocks / (waves x resident slots)) among those leaving at least min_chunk
// planes per block; the smaller split wins ties.
int best_zsplit(int tiles, int slots, int nz, int min_chunk) {
  int best = 1;
  double best_eff = -1.0;
  const int maxz = nz / min_chunk > 1 ? nz / min_chunk : 1;
  for (int zs = 1; zs <= maxz; ++zs) {
    const int kc = (nz + zs - 1) / zs;
    const int z = (nz + kc - 1) / kc;
    const long long blocks = (long long)tiles * z;
    const long long waves = (blocks + slots - 1) / slots;
    const double eff = (double)blocks / (double)(waves * slots);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = z;
    }
  }
  return best;
}

Geom make_geom(int nx, int ny, int nz) {
  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.Px = roundup(nx + 1, 8);
  g.Py = ny + 1;
  g.sz = (i64)g.Px * g.Py;
  // one pad plane and two pad rows in front (index (-1,-1,-1) = Px - 1 >= 0);
  // off and len are multiples of Px so the arrays are 2-D tensors of rows
  g.off = g.sz + 2 * (i64)g.Px;
  g.len = g.off + (i64)(nz + 1) * g.sz + g.Px;
  return g;
}

int lin_blocks(const mg_handle* h, i64 n) {
  i64 b = (n + 255) / 256;
  i64 cap = (i64)h->nsm * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Launch on the handle's stream, as a programmatic dependent launch when the
// handle enables it (the kernel's first action is griddepcontrol.wait).
template <class... KArgs, class... Args>
void launch(const mg_handle* h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args);

template <class T> mg_status alloc(mg_handle* h, T** p, i64 n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MG_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(q);
  e = cudaMemsetAsync(q, 0, (size_t)n * sizeof(T), h->s);
  if (e != cudaSuccess) return fail(h, MG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  *p = (T*)q;
  return MG_OK;
}
#define AL(ptr, T, n)                                  \
  do {                                                 \
    T* t_ = nullptr;                                   \
    mg_status s_ = alloc<T>(h, &t_, (n));              \
    if (s_ != MG_OK) return s_;                        \
    ptr = t_;                                          \
  } while (0)

// ---- TMA tensor maps ---------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tma_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

template <class T> CUtensorMapDataType tma_dtype();
template <> CUtensorMapDataType tma_dtype<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <> CUtensorMapDataType tma_dtype<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tma_dtype<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

// 2-D view of a padded level array: rows of Px elements; box bw x bh elements.
template <class T> bool tma_encode(CUtensorMap* m, const void* base, const Geom& g, int bw, int bh) {
  EncodeTiledFn fn = tma_encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)g.Px, (cuuint64_t)(g.len / g.Px)};
  const cuuint64_t strides[1] = {(cuuint64_t)g.Px * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, tma_dtype<T>(), 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// ---- opt-in kernel timing: event pairs around launches, collected at sync points
constexpr int EV_POOL = 2048;

int tm_begin(mg_handle* h, int cls, int level) {
  if (!h->timing || h->ev_next + 2 > (int)h->evpool.size()) return -1;
  if (!((h->t_cls_mask >> cls) & 1) || !((h->t_lvl_mask >> level) & 1)) return -1;
  const int e = h->ev_next;
  h->ev_next += 2;
  cudaEventRecordWithFlags(h->evpool[e], h->s, h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  return e;
}

void tm_end(mg_handle* h, int e, int cls, int level, double pts) {
  if (e < 0) return;
  cudaEventRecordWithFlags(h->evpool[e + 1], h->s, h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  mg_handle::TRec r{cls, level, pts, e};
  if (h->capturing) h->graph_recs.push_back(r);
  else h->pending.push_back(r);
}

void tm_collect(mg_handle* h) {
  if (!h->timing) return;
  for (const auto& r : h->pending) {
    float ms = 0.f;
    cudaEventSynchronize(h->evpool[r.ev + 1]);  // launches queued after the last host sync may still run
    if (cudaEventElapsedTime(&ms, h->evpool[r.ev], h->evpool[r.ev + 1]) == cudaSuccess) {
      h->t_ms[r.cls][r.level] += ms;
      h->t_n[r.cls][r.level] += 1;
      h->t_pts[r.cls][r.level] += r.pts;
    } else {
      cudaGetLastError();
    }
  }
  h->pending.clear();
  h->ev_next = h->ev_graph_end;
}

// z-marching launch geometry: 32x4 column tiles; the planes are split into
// chunks of at least 2 with the best wave efficiency over 8 resident blocks
// per SM (small levels simply get fewer blocks).
dim3 zm_grid(const mg_handle* h, const Geom& g, int* kchunk) {
  dim3 grid((g.nx + ZM_TX - 1) / ZM_TX, (g.ny + ZM_TY - 1) / ZM_TY, 1);
  const int zs = best_zsplit(grid.x * grid.y, h->nsm * 8, g.nz, 2);
  const int kc = (g.nz + zs - 1) / zs;
  grid.z = (g.nz + kc - 1) / kc;
  *kchunk = kc;
  return grid;
}

// Plane chunks as short as one plane: on the small coarse levels a wave is
// latency-bound and more, shorter chunks finish sooner (measured at 257^3:
// levels 2 and 3 take 13% and 19% less than with chunks of at least 2).
dim3 zv_grid(const mg_handle* h, const Geom& g, int* kchunk) {
  dim3 grid((g.nx + ZV_TX - 1) / ZV_TX, (g.ny + ZV_TY - 1) / ZV_TY, 1);
  const int zs = best_zsplit(grid.x * grid.y, h->nsm * 8, g.nz, 1);
  const int kc = (g.nz + zs - 1) / zs;
  grid.z = (g.nz + kc - 1) / kc;
  *kchunk = kc;
  return grid;
}

// One z-marching pass of a point operation over level geometry g: stencil
// operations, the prolongation and the restriction go to the two-points-per-
// thread kernels unless the scalar driver was asked for (the float64 CG
// operator and the 27-point operators always use the scalar driver).

// The operand of a stencil or transfer pass whose z neighbours (the pad
// planes, which hold the neighbours' planes in a z-slab) it reads; pointwise
// passes have none.
template <class Op> struct HaloOf {
  static void* ptr(const Op&) { return nullptr; }
  static int bytes() { return 0; }
  static Geom geom(const Op&, const Geom& g) { return g; }
};
#define MG_HALO_OF(TPL, OPT, EXPR, TVT, GEXPR)                                \
  template <TPL> struct HaloOf<OPT> {                                         \
    static void* ptr(const OPT& op) { return (void*)(EXPR); }                 \
    static int bytes() { return (int)sizeof(TVT); }                          \
    static Geom geom(const OPT& op, const Geom& g) { return GEXPR; }          \
  };
#define MG_COMMA ,
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpApply<R MG_COMMA TV MG_COMMA TC>, op.u, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpChebStep<R MG_COMMA TV MG_COMMA TC>, op.x, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpChebStepDot<R MG_COMMA TV MG_COMMA TC>, op.step.x, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpChebZero<R MG_COMMA TV MG_COMMA TC>, op.b, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TB MG_COMMA class TC,
           OpResidual<R MG_COMMA TV MG_COMMA TB MG_COMMA TC>, op.x, TV, g)
MG_HALO_OF(class R MG_COMMA class TV, OpRestrict<R MG_COMMA TV>, op.r, TV, op.gf)
MG_HALO_OF(class R MG_COMMA class TV, OpProlong<R MG_COMMA TV>, op.e, TV, op.gc)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpApply27<R MG_COMMA TV MG_COMMA TC>, op.u, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpChebZero27<R MG_COMMA TV MG_COMMA TC>, op.b, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TC, OpChebStep27<R MG_COMMA TV MG_COMMA TC>, op.x, TV, g)
MG_HALO_OF(class R MG_COMMA class TV MG_COMMA class TB MG_COMMA class TC,
           OpResidual27<R MG_COMMA TV MG_COMMA TB MG_COMMA TC>, op.x, TV, g)
#undef MG_HALO_OF
#undef MG_COMMA
template <class TB> struct HaloOf<OpResidualD<TB>> {
  static void* ptr(const OpResidualD<TB>& op) { return (void*)op.x; }
  static int bytes() { return 8; }
  static Geom geom(const OpResidualD<TB>&, const Geom& g) { return g; }
};
template <> struct HaloOf<OpApplyPQ> {
  static void* ptr(const OpApplyPQ& op) { return (void*)op.p; }
  static int bytes() { return 8; }
  static Geom geom(const OpApplyPQ&, const Geom& g) { return g; }
};

template <class Op> void set_halo(const mg_handle* h, const Op& op, const Geom& g) {
  if (!h->rec) return;
  h->halo_ptr = HaloOf<Op>::ptr(op);
  h->halo_bytes = HaloOf<Op>::bytes();
  h->halo_g = HaloOf<Op>::geom(op, g);
}

template <class R, class TV> void zv_xfer(mg_handle* h, const Geom& gc, const OpRestrict<R, TV>& op) {
  int kc;
  dim3 grid = zv_grid(h, gc, &kc);
  launch(h, k_restrict_v<R, TV>, grid, dim3(ZV_THREADS), 0, op, gc, kc);
}
template <class R, class TV> void zv_xfer(mg_handle* h, const Geom& g, const OpProlong<R, TV>& op) {
  dim3 grid((g.nx + 255) / 256, (g.ny + 3) / 4, g.nz);
  launch(h, k_prolong_v<R, TV>, grid, dim3(PV_THREADS), 0, op, g);
}

template <bool RED, class Op>
int zmarch(mg_handle* h, const Geom& g, const Op& op, int cls = -1, int level = 0) {
  int kc;
  set_halo(h, op, g);
  if constexpr (ZvXfer<Op>::ok) {  // prolongation / restriction: vector kernels
    if (h->zvec) {
      const int e = cls >= 0 ? tm_begin(h, cls, level) : -1;
      zv_xfer(h, g, op);
      ++h->launches;
      tm_end(h, e, cls, level, (double)g.npts());
      return 0;
    }
  }
  if constexpr (Zv<Op>::ok) {
    if (h->zvec) {
      dim3 grid = zv_grid(h, g, &kc);
      const int e = cls >= 0 ? tm_begin(h, cls, level) : -1;
      launch(h, k_zvec<Op, RED>, grid, dim3(ZV_THREADS), 0, op, g, kc, h->partials, h->pstride);
      ++h->launches;
      tm_end(h, e, cls, level, (double)g.npts());
      return grid.x * grid.y * grid.z;
    }
  }
  dim3 grid = zm_grid(h, g, &kc);
  const int e = cls >= 0 ? tm_begin(h, cls, level) : -1;
  launch(h, k_zmarch<Op, RED>, grid, dim3(ZM_THREADS), 0, op, g, kc, h->partials, h->pstride);
  ++h->launches;
  tm_end(h, e, cls, level, (double)g.npts());
  return grid.x * grid.y * grid.z;
}

// Pointwise pass over n elements of the finest level: one wave of the kernel's
// own resident blocks (a grid-stride loop over more blocks than fit at once
// would leave a partial second wave).
template <bool RED, class Op> int linear(mg_handle* h, i64 n, const Op& op, int cls = -1) {
  i64 lo = 0;
  if (h->lin_hi >= 0) {  // a slab: its interior planes only
    lo = h->lin_lo;
    n = h->lin_hi;
  }
  static int per_sm = 0;  // per instantiation: resident blocks per SM
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_linear<Op, RED>, LIN_THREADS, 0) != cudaSuccess || v < 1)
      v = 4;
    per_sm = v;
  }
  const i64 want = ((n - lo) / 4 + LIN_THREADS - 1) / LIN_THREADS;
  const i64 wave = (i64)h->nsm * per_sm;
  int nb = (int)(want < wave ? want : wave);
  if (nb < 1) nb = 1;
  if (nb > h->lin_grid) nb = h->lin_grid;
  const int e = cls >= 0 ? tm_begin(h, cls, 0) : -1;
  launch(h, k_linear<Op, RED>, dim3(nb), dim3(LIN_THREADS), 0, op, lo, n, h->partials, h->pstride);
  ++h->launches;
  tm_end(h, e, cls, 0, (double)h->lv[0].g.npts());
  return nb;
}

void finish(mg_handle* h, int nblocks, int mode, Scal* mirror = nullptr) {
  if (h->rec) {  // a slab: the reduction is finished across the slabs at replay
    Pass ps;
    ps.kind = Pass::FINISH;
    ps.nb = nblocks;
    ps.mode = mode;
    h->rec->push_back(ps);
    return;
  }
  int flex = h->prm.flexible;
  launch(h, k_finish, dim3(1), dim3(FIN_THREADS), 0, (const double*)h->partials, nblocks, h->pstride, mode, h->dsc, flex,
         mirror);
  ++h->launches;
}

int sweep_flips(int degree, bool zero) { return zero ? (degree == 1 ? 1 : degree - 1) : degree; }

// Buffer index holding a level's result after pre- and post-smoothing.
int level_result_cur(const mg_params& p) {
  int f = 0;
  for (int s = 0; s < p.nu_pre; ++s) f += sweep_flips(p.cheby_degree, s == 0);
  for (int s = 0; s < p.nu_post; ++s) f += sweep_flips(p.cheby_degree, false);
  return f & 1;
}

void cheb_consts(const mg_params& p, double beta_l, double alpha_l, double* theta, double* delta, double* sigma) {
  if (p.smoother == MG_SMOOTHER_RICHARDSON) {  // one step x += omega D^-1 (b - A x) per sweep
    *theta = 1.0 / p.richardson_omega;
    *delta = *sigma = 0.0;
    return;
  }
  const double beta = beta_l, alpha = alpha_l;
  *theta = 0.5 * (beta + alpha);
  *delta = 0.5 * (beta - alpha);
  *sigma = *theta / *delta;
}

// Coefficients of the Chebyshev steps j = 1..degree-1 (the same for every
// sweep: the recurrence always restarts from rho_0 = 1/sigma), and 1/theta.
void cheb_table(const mg_params& p, double beta_l, double alpha_l, double* inv_theta, double* c1, double* c2) {
  double theta, delta, sigma;
  cheb_consts(p, beta_l, alpha_l, &theta, &delta, &sigma);
  *inv_theta = 1.0 / theta;
  double rho_prev = 1.0 / sigma;
  c1[0] = c2[0] = 0.0;
  for (int j = 1; j < p.cheby_degree; ++j) {
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    c1[j] = rho * rho_prev;
    c2[j] = 2.0 * rho / delta;
    rho_prev = rho;
  }
}

mg_status read_scal(mg_handle* h);

template <class TV, class TC> struct Impl {
  using TVt = TV;
  using TCt = TC;
  static TV* V(void* p) { return (TV*)p; }
  static const TC* C(void* p) { return (const TC*)p; }

  // ---- TMA-staged stencil launches -------------------------------------------
  template <int KIND, bool HAS_D, bool DOT> static void tma_attr(mg_handle* h) {
    using Lay = TmaLayout<KIND, HAS_D, DOT, TV, TC>;
    cudaFuncSetAttribute(k_tma_stencil<KIND, HAS_D, DOT, TV, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Lay::SMEM);
  }

  // Encodes the tensor maps of level l and fixes its launch geometry.
  static bool tma_prepare(mg_handle* h, int l) {
    LevelBuf& Lv = h->lv[l];
    const Geom& g = Lv.g;
    constexpr int BWV = XHalo<TV>::BW, BWC = XHalo<TC>::BW;
    bool ok = true;
    for (int c = 0; c < 2; ++c) ok = ok && tma_encode<TV>(&Lv.m_full_x[c], Lv.x[c], g, BWV, TT_Y + 2);
    ok = ok && tma_encode<TV>(&Lv.m_full_b, Lv.b, g, BWV, TT_Y + 2);
    ok = ok && tma_encode<TV>(&Lv.m_full_dinv, Lv.dinv, g, BWV, TT_Y + 2);
    ok = ok && tma_encode<TC>(&Lv.m_kx, Lv.kx, g, BWC, TT_Y);
    ok = ok && tma_encode<TC>(&Lv.m_ky, Lv.ky, g, TT_X, TT_Y + 1);
    ok = ok && tma_encode<TC>(&Lv.m_kz, Lv.kz, g, TT_X, TT_Y);
    ok = ok && tma_encode<TV>(&Lv.m_c_dinv, Lv.dinv, g, TT_X, TT_Y);
    ok = ok && tma_encode<TV>(&Lv.m_c_b, Lv.b, g, TT_X, TT_Y);
    ok = ok && tma_encode<TV>(&Lv.m_c_d, Lv.d, g, TT_X, TT_Y);
    if (!ok) return false;
    // grid: 32x8 tiles; planes split so that about one wave of blocks is
    // resident (shared memory bounds the blocks per SM)
    const int gx = (g.nx + TT_X - 1) / TT_X, gy = (g.ny + TT_Y - 1) / TT_Y;
    tma_attr<TK_STEP, true, true>(h);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tma_stencil<TK_STEP, true, true, TV, TC>, TT_THREADS,
                                                  TmaLayout<TK_STEP, true, true, TV, TC>::SMEM);
    per_sm = per_sm < 1 ? 1 : per_sm;
    // whole waves only: the largest plane split whose blocks all fit at once
    int zs = (h->nsm * per_sm) / (gx * gy);
    zs = zs < 1 ? 1 : (zs > g.nz ? g.nz : zs);
    const int kc = (g.nz + zs - 1) / zs;
    Lv.tma_kchunk = kc;
    Lv.tma_grid[0] = gx;
    Lv.tma_grid[1] = gy;
    Lv.tma_grid[2] = (g.nz + kc - 1) / kc;
    tma_attr<TK_ZERO, false, false>(h);
    tma_attr<TK_STEP, false, false>(h);
    tma_attr<TK_STEP, true, false>(h);
    tma_attr<TK_STEP, false, true>(h);
    tma_attr<TK_STEP, true, true>(h);
    tma_attr<TK_RESID, false, false>(h);
    Lv.tma = true;
    return true;
  }

  template <int KIND, bool HAS_D, bool DOT>
  static int tma_launch(mg_handle* h, int l, const CUtensorMap& f0, const CUtensorMap* f1, TV* xout, TV* dout,
                        double c1, double c2, double inv_theta, int cls) {
    LevelBuf& Lv = h->lv[l];
    TmaMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    maps.m[0] = f0;
    if (f1) maps.m[1] = *f1;
    maps.m[2] = Lv.m_kx;
    maps.m[3] = Lv.m_ky;
    maps.m[4] = Lv.m_kz;
    maps.m[5] = Lv.m_c_dinv;
    maps.m[6] = Lv.m_c_b;
    maps.m[7] = Lv.m_c_d;
    TmaArgs<TV, TC> a{};
    a.g = Lv.g;
    a.kchunk = Lv.tma_kchunk;
    a.rowbase = (int)(Lv.g.off / Lv.g.Px);
    a.xout = xout;
    a.dout = dout;
    a.kx = C(Lv.kx);
    a.c1 = (float)c1;
    a.c2 = (float)c2;
    a.inv_theta = (float)inv_theta;
    a.dc1 = c1;
    a.dc2 = c2;
    a.dinv_theta = inv_theta;
    a.partials = h->partials;
    a.status = &h->dsc->status;
    a.poll_limit = h->prm.test_inject == 3 ? 0 : TMA_POLL_LIMIT;
    using Lay = TmaLayout<KIND, HAS_D, DOT, TV, TC>;
    dim3 grid(Lv.tma_grid[0], Lv.tma_grid[1], Lv.tma_grid[2]);
    const int e = tm_begin(h, cls, l);
    launch(h, k_tma_stencil<KIND, HAS_D, DOT, TV, TC>, grid, dim3(TT_THREADS), Lay::SMEM, maps, a);
    ++h->launches;
    tm_end(h, e, cls, l, (double)Lv.g.npts());
    return grid.x * grid.y * grid.z;
  }

  // Chebyshev steps j_from..degree-1 of one sweep on level l: the iterate is in
  // buffer cur (and d_{j_from-1} in Lv.d when j_from > 0), rho_prev = rho_{j_from-1}.
  // With fuse_rz the last step also accumulates rho = b.z for the outer CG and
  // finishes the CG scalars.  Returns the buffer holding the result.
  static int cheb_steps(mg_handle* h, int l, int cur, int j_from, double rho_prev, bool fuse_rz) {
    LevelBuf& Lv = h->lv[l];
    const mg_params& p = h->prm;
    double theta, delta, sigma;
    cheb_consts(p, Lv.beta, Lv.alpha, &theta, &delta, &sigma);
    const TV inv_theta = (TV)(1.0 / theta);
    for (int j = j_from; j < p.cheby_degree; ++j) {
      double c1 = 0.0, c2 = 0.0;
      if (j > 0) {
        const double rho = 1.0 / (2.0 * sigma - rho_prev);
        c1 = rho * rho_prev;
        c2 = 2.0 * rho / delta;
        rho_prev = rho;
      }
      const bool dot = fuse_rz && j + 1 == p.cheby_degree;
      TV* xo = V(Lv.x[cur ^ 1]);
      TV* dout = j + 1 < p.cheby_degree ? V(Lv.d) : nullptr;
      const TV* dprev = j > 0 ? V(Lv.d) : nullptr;
      int nb = -1;
      if (Lv.tma) {
        const CUtensorMap& f0 = Lv.m_full_x[cur];
        if (j > 0 && dot) nb = tma_launch<TK_STEP, true, true>(h, l, f0, nullptr, xo, dout, c1, c2, 1.0 / theta, MG_K_CHEB_STEP);
        else if (j > 0) tma_launch<TK_STEP, true, false>(h, l, f0, nullptr, xo, dout, c1, c2, 1.0 / theta, MG_K_CHEB_STEP);
        else if (dot) nb = tma_launch<TK_STEP, false, true>(h, l, f0, nullptr, xo, dout, c1, c2, 1.0 / theta, MG_K_CHEB_STEP);
        else tma_launch<TK_STEP, false, false>(h, l, f0, nullptr, xo, dout, c1, c2, 1.0 / theta, MG_K_CHEB_STEP);
      } else if (Lv.g27) {  // Galerkin levels are never the finest, so no fused dot
        OpChebStep27<TV, TV, TC> op{V(Lv.x[cur]), dprev, V(Lv.b), V(Lv.dinv), xo, dout, C(Lv.w), Lv.g.len,
                                    (TV)c1, (TV)c2, inv_theta};
        zmarch<false>(h, Lv.g, op, MG_K_CHEB_STEP, l);
      } else {
        OpChebStep<TV, TV, TC> op{V(Lv.x[cur]), dprev, V(Lv.b), V(Lv.dinv), xo, dout, C(Lv.kx), C(Lv.ky), C(Lv.kz),
                                  (TV)c1, (TV)c2, inv_theta};
        if (dot) nb = zmarch<true>(h, Lv.g, OpChebStepDot<TV, TV, TC>{op}, MG_K_CHEB_STEP, l);
        else zmarch<false>(h, Lv.g, op, MG_K_CHEB_STEP, l);
      }
      if (dot) {
        finish(h, nb, FIN_RZ);
        h->rz_fused = true;
      }
      cur ^= 1;
    }
    return cur;
  }

  // One smoother sweep on level l starting from buffer cur; returns the new cur.
  // With fuse_rz the last step also accumulates rho = b.z for the outer CG.
  static int sweep(mg_handle* h, int l, int cur, bool zero, bool fuse_rz = false) {
    LevelBuf& Lv = h->lv[l];
    const mg_params& p = h->prm;
    double theta, delta, sigma;
    cheb_consts(p, Lv.beta, Lv.alpha, &theta, &delta, &sigma);
    const TV inv_theta = (TV)(1.0 / theta);
    if (!zero) return cheb_steps(h, l, cur, 0, 1.0 / sigma, fuse_rz);
    if (p.cheby_degree == 1) {
      OpChebZero1<TV, TV> op{V(Lv.b), V(Lv.dinv), V(Lv.x[cur ^ 1]), inv_theta};
      zmarch<false>(h, Lv.g, op, MG_K_CHEB_ZERO, l);
      return cur ^ 1;
    }
    if constexpr (std::is_same<TV, double>::value) {
      if (!Lv.tma) {  // store step 0, then step 1 as an ordinary step (OpChebStart)
        OpChebStart<TV, TV> op{V(Lv.b), V(Lv.dinv), V(Lv.x[cur]), V(Lv.d), inv_theta};
        zmarch<false>(h, Lv.g, op, MG_K_CHEB_ZERO, l);
        return cheb_steps(h, l, cur, 1, 1.0 / sigma, fuse_rz);
      }
    }
    const double rho_prev = 1.0 / sigma;
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    const double c1 = rho * rho_prev, c2 = 2.0 * rho / delta;
    TV* dout = p.cheby_degree > 2 ? V(Lv.d) : nullptr;
    if (Lv.tma) {
      tma_launch<TK_ZERO, false, false>(h, l, Lv.m_full_b, &Lv.m_full_dinv, V(Lv.x[cur ^ 1]), dout, c1, c2,
                                        1.0 / theta, MG_K_CHEB_ZERO);
    } else if (Lv.g27) {
      OpChebZero27<TV, TV, TC> op{V(Lv.b), V(Lv.dinv), V(Lv.x[cur ^ 1]), dout, C(Lv.w), Lv.g.len,
                                  (TV)c1, (TV)c2, inv_theta};
      zmarch<false>(h, Lv.g, op, MG_K_CHEB_ZERO, l);
    } else {
      OpChebZero<TV, TV, TC> op{V(Lv.b), V(Lv.dinv), V(Lv.x[cur ^ 1]), dout, C(Lv.kx), C(Lv.ky), C(Lv.kz),
                                (TV)c1, (TV)c2, inv_theta};
      zmarch<false>(h, Lv.g, op, MG_K_CHEB_ZERO, l);
    }
    return cheb_steps(h, l, cur ^ 1, 2, rho, fuse_rz);
  }

  // Coarse-grid correction x += P e followed by the post-smoothing sweeps of
  // level l.
  static int correct_and_post_smooth(mg_handle* h, int l, int cur, int ccur, bool fuse_rz) {
    LevelBuf& Lv = h->lv[l];
    LevelBuf& Cv = h->lv[l + 1];
    const mg_params& p = h->prm;
    OpProlong<TV, TV> pr{Cv.g, V(Cv.x[ccur]), V(Lv.x[cur])};
    zmarch<false>(h, Lv.g, pr, MG_K_PROLONG, l);
    for (int s = 0; s < p.nu_post; ++s) cur = sweep(h, l, cur, false, fuse_rz && s + 1 == p.nu_post);
    return cur;
  }

  // whether a cluster of nb bottom-kernel blocks can be resident at once
  static bool bottom_cluster_fits(int nb) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(BOT_THREADS);
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = nb;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, k_bottom<TV, TV, TC, true>, &cfg) == cudaSuccess && n > 0;
    cudaGetLastError();
    return ok;
  }

  static void bottom(mg_handle* h, int l0) {
    if (h->rec) {  // a slab reached the agglomeration level: the root takes over at replay
      Pass ps;
      ps.kind = Pass::AGGLOM;
      ps.level = l0;
      h->rec->push_back(ps);
      return;
    }
    BotArgs<TV, TC> a{};
    a.nlev = h->L - l0;
    for (int l = l0; l < h->L; ++l) {
      LevelBuf& Lv = h->lv[l];
      BotLevel<TV, TC>& B = a.lv[l - l0];
      B.g = Lv.g;
      B.x[0] = V(Lv.x[0]);
      B.x[1] = V(Lv.x[1]);
      B.d = V(Lv.d);
      B.b = V(Lv.b);
      B.r = V(Lv.r);
      B.dinv = V(Lv.dinv);
      B.kx = C(Lv.kx);
      B.ky = C(Lv.ky);
      B.kz = C(Lv.kz);
      B.w = Lv.g27 ? C(Lv.w) : nullptr;
      B.dg = Lv.g27 ? V(Lv.dg) : nullptr;
      double it, c1[BOT_MAXDEG], c2[BOT_MAXDEG];
      cheb_table(h->prm, Lv.beta, Lv.alpha, &it, c1, c2);
      B.inv_theta = (TV)it;
      for (int j = 0; j < h->prm.cheby_degree; ++j) {
        B.c1[j] = (TV)c1[j];
        B.c2[j] = (TV)c2[j];
      }
    }
    a.nu_pre = h->prm.nu_pre;
    a.nu_post = h->prm.nu_post;
    a.degree = h->prm.cheby_degree;
    a.Lc = h->Lc;
    a.Li = h->Li;
    a.Ac = h->prm.coarse_solve == 1 ? h->Ac : nullptr;
    a.coarse_rtol = h->prm.coarse_rtol;
    a.coarse_maxit = h->prm.coarse_maxit;
    a.nc = h->nc;
    const int e = tm_begin(h, MG_K_BOTTOM, l0);
    if (h->bot_cluster > 1)
      launch_cluster(h, k_bottom<TV, TV, TC, true>, h->bot_cluster, dim3(BOT_THREADS), a);
    else
      launch(h, k_bottom<TV, TV, TC, false>, dim3(1), dim3(BOT_THREADS), 0, a);
    ++h->launches;
    tm_end(h, e, MG_K_BOTTOM, l0, (double)h->lv[l0].g.npts());
  }

  // r = b - A x[cur] on level l, then b of level l+1 = R r.
  static void residual_restrict(mg_handle* h, int l, int cur) {
    LevelBuf& Lv = h->lv[l];
    LevelBuf& Cv = h->lv[l + 1];
    if (Lv.tma) {
      tma_launch<TK_RESID, false, false>(h, l, Lv.m_full_x[cur], nullptr, V(Lv.r), nullptr, 0.0, 0.0, 0.0,
                                         MG_K_RESID);
    } else if (Lv.g27) {
      OpResidual27<TV, TV, TV, TC> res{V(Lv.x[cur]), V(Lv.b), V(Lv.r), C(Lv.w), Lv.g.len, V(Lv.dg)};
      zmarch<false>(h, Lv.g, res, MG_K_RESID, l);
    } else if (std::is_same<TV, double>::value && l == 0 && !h->rec && !h->sub) {
      // float64 form, finest level: the stored float64 diagonal
      OpResidualD<double> res{(const double*)Lv.x[cur], (const double*)Lv.b, (double*)Lv.r, h->dg64,
                              (const double*)Lv.kx, (const double*)Lv.ky, (const double*)Lv.kz};
      zmarch<false>(h, Lv.g, res, MG_K_RESID, l);
    } else {
      OpResidual<TV, TV, TV, TC> res{V(Lv.x[cur]), V(Lv.b), V(Lv.r), C(Lv.kx), C(Lv.ky), C(Lv.kz)};
      zmarch<false>(h, Lv.g, res, MG_K_RESID, l);
    }
    OpRestrict<TV, TV> rs{Lv.g, V(Lv.r), V(Cv.b)};
    zmarch<false>(h, Cv.g, rs, MG_K_RESTRICT, l);
  }

  // V-cycle from level l with zero initial guess; b of level l must be set.
  // Returns the buffer index of level l holding the result.
  static int vcycle(mg_handle* h, int l, bool fuse_rz = false) {
    if (l >= h->lb) {
      bottom(h, l);
      return l == h->L - 1 ? 0 : level_result_cur(h->prm);
    }
    LevelBuf& Lv = h->lv[l];
    int cur = 0;
    for (int s = 0; s < h->prm.nu_pre; ++s) cur = sweep(h, l, cur, s == 0);
    if (h->prm.nu_pre == 0) {
      void* x0 = Lv.x[0];
      const size_t bytes = (size_t)Lv.g.len * sizeof(TV);
      cudaStream_t st = h->s;
      if (h->rec) {
        Pass ps;
        ps.kind = Pass::MEMSET;
        ps.fn = [x0, bytes, st]() { cudaMemsetAsync(x0, 0, bytes, st); };
        h->rec->push_back(std::move(ps));
      } else {
        cudaMemsetAsync(x0, 0, bytes, st);
      }
    }
    residual_restrict(h, l, cur);
    const int ccur = vcycle(h, l + 1);
    return correct_and_post_smooth(h, l, cur, ccur, fuse_rz);
  }

  // z = M^-1 r; the finest right-hand side b (the float64 residual, or its
  // float32 copy in the mixed forms) must be in place.  Ends with rho = b.z
  // (OpChebStepDot) and the CG beta in the scalar block.  Returns the level-0
  // buffer (type TV) holding z.
  static TV* precondition(mg_handle* h) {
    LevelBuf& L0 = h->lv[0];
    h->rz_fused = false;
    const int zc = vcycle(h, 0, true);
    if (!h->rz_fused) {
      const int nb = linear<true>(h, L0.g.len, LinDotT<TV>{V(L0.b), V(L0.x[zc])}, MG_K_DOT);
      finish(h, nb, FIN_RZ);
    }
    return V(L0.x[zc]);
  }

  // Largest eigenvalue of D^-1 A on level l: CG with the Jacobi preconditioner
  // for 10 steps from a seeded random right-hand side, in the V-cycle
  // precision; the CG coefficients give the Lanczos tridiagonal matrix
  // (T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_{j,j+1} = sqrt(b_j)/a_j), whose largest
  // eigenvalue is found by bisection on Sturm counts.  Runs at setup in the
  // level's work vectors.
  static mg_status lanczos(mg_handle* h, int l, double* lmax) {
    LevelBuf& Lv = h->lv[l];
    const Geom& g = Lv.g;
    const i64 n = g.len;
    TV *r = V(Lv.r), *z = V(Lv.d), *p = V(Lv.x[0]), *q = V(Lv.x[1]);
    const TV* dinv = V(Lv.dinv);
    const int lb = lin_blocks(h, n);
    mg_status s;
    auto dot = [&](const TV* a, const TV* b, double* out) -> mg_status {
      const int nb = linear<true>(h, n, LinDotT<TV>{a, b});
      finish(h, nb, FIN_BB);
      mg_status st = read_scal(h);
      *out = h->hsc->bb;
      return st;
    };
    k_lz_fill<TV><<<lin_blocks(h, g.npts()), 256, 0, h->s>>>(r, g, 20160424ull);
    k_lz_jacobi<TV><<<lb, 256, 0, h->s>>>(z, r, dinv, n);
    CK(cudaMemcpyAsync(p, z, (size_t)n * sizeof(TV), cudaMemcpyDeviceToDevice, h->s));
    double rz;
    if ((s = dot(r, z, &rz)) != MG_OK) return s;
    double a[10], b[10];
    int m = 0;
    for (int j = 0; j < 10 && j < g.npts(); ++j) {
      if (Lv.g27) zmarch<false>(h, g, OpApply27<TV, TV, TC>{p, q, C(Lv.w), g.len, V(Lv.dg)});
      else zmarch<false>(h, g, OpApply<TV, TV, TC>{p, q, C(Lv.kx), C(Lv.ky), C(Lv.kz)});
      double pq;
      if ((s = dot(p, q, &pq)) != MG_OK) return s;
      if (!(pq > 0.0) || !(rz > 0.0)) break;
      a[j] = rz / pq;
      k_lz_axpy<TV><<<lb, 256, 0, h->s>>>(r, q, -a[j], n);
      k_lz_jacobi<TV><<<lb, 256, 0, h->s>>>(z, r, dinv, n);
      double rz_new;
      if ((s = dot(r, z, &rz_new)) != MG_OK) return s;
      b[j] = rz_new / rz;
      k_lz_xpay<TV><<<lb, 256, 0, h->s>>>(p, z, b[j], n);
      rz = rz_new;
      m = j + 1;
    }
    CKL();
    if (m == 0) {
      *lmax = 2.0;
      return MG_OK;
    }
    double d[10], e[10];
    for (int j = 0; j < m; ++j) {
      d[j] = 1.0 / a[j] + (j > 0 ? b[j - 1] / a[j - 1] : 0.0);
      e[j] = j + 1 < m ? std::sqrt(b[j]) / a[j] : 0.0;
    }
    // Gershgorin bracket, then bisection on the number of eigenvalues below x
    double lo = d[0], hi = d[0];
    for (int j = 0; j < m; ++j) {
      const double rad = std::fabs(e[j]) + (j > 0 ? std::fabs(e[j - 1]) : 0.0);
      lo = std::min(lo, d[j] - rad);
      hi = std::max(hi, d[j] + rad);
    }
    auto below = [&](double x) {
      int c = 0;
      double piv = 1.0;
      for (int j = 0; j < m; ++j) {
        piv = d[j] - x - (j > 0 ? e[j - 1] * e[j - 1] / piv : 0.0);
        if (piv == 0.0) piv = -1e-300;
        c += piv < 0.0;
      }
      return c;
    };
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (below(mid) >= m) hi = mid;
      else lo = mid;
    }
    *lmax = hi;
    return MG_OK;
  }

  // float32 copy of the float64 residual as the V-cycle's finest right-hand side
  static void cast_rhs(mg_handle* h) {
    LevelBuf& L0 = h->lv[0];
    if (h->prm.precision == MG_FP64) return;
    const int e = tm_begin(h, MG_K_CAST, 0);
    launch(h, k_cast<TV, double>, dim3(lin_blocks(h, L0.g.len)), dim3(256), 0, (const double*)h->cr, V(L0.b),
           L0.g.len);
    ++h->launches;
    tm_end(h, e, MG_K_CAST, 0, (double)L0.g.npts());
  }
};

template <class F> auto dispatch(mg_handle* h, F&& f) {
  switch (h->prm.precision) {
    case MG_MIXED_FP32: return f(Impl<float, float>{});
    case MG_MIXED_BF16K: return f(Impl<float, __nv_bfloat16>{});
    default: return f(Impl<double, double>{});
  }
}

size_t vbytes(const mg_handle* h) { return h->prm.precision == MG_FP64 ? 8 : 4; }
size_t cbytes(const mg_handle* h) {
  return h->prm.precision == MG_FP64 ? 8 : (h->prm.precision == MG_MIXED_FP32 ? 4 : 2);
}

mg_status sync_check(mg_handle* h) {
  CKL();
  CK(cudaStreamSynchronize(h->s));
  return MG_OK;
}

mg_status read_scal(mg_handle* h) {
  CKL();
  CK(cudaMemcpyAsync(h->hsc, h->dsc, sizeof(Scal), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  tm_collect(h);
  return MG_OK;
}

// The same read in two halves, so that more work can be queued behind it
// before the host waits.  The outer iteration's last reduction has already
// written the scalars to the host (k_finish's mirror), so only an event is
// queued; otherwise a copy.
mg_status read_scal_issue(mg_handle* h, bool mirrored) {
  CKL();
  if (!mirrored) CK(cudaMemcpyAsync(h->hsc, h->dsc, sizeof(Scal), cudaMemcpyDeviceToHost, h->s));
  CK(cudaEventRecord(h->ev_scal, h->s));
  return MG_OK;
}
mg_status read_scal_wait(mg_handle* h) {
  CK(cudaEventSynchronize(h->ev_scal));
  tm_collect(h);
  return MG_OK;
}

// pack a dense float64 nodal array into a padded buffer of the level's vector type
mg_status pack_level(mg_handle* h, int l, const double* src, void* dst, bool f64) {
  const Geom& g = h->lv[l].g;
  const int nb = lin_blocks(h, g.npts());
  if (f64 || h->prm.precision == MG_FP64) k_pack<double><<<nb, 256, 0, h->s>>>(src, (double*)dst, g);
  else k_pack<float><<<nb, 256, 0, h->s>>>(src, (float*)dst, g);
  ++h->launches;
  CKL();
  return MG_OK;
}

mg_status unpack_level(mg_handle* h, int l, const void* src, double* dst, bool f64) {
  const Geom& g = h->lv[l].g;
  const int nb = lin_blocks(h, (i64)(g.nx + 2) * (g.ny + 2) * (g.nz + 2));
  if (f64 || h->prm.precision == MG_FP64) k_unpack<double><<<nb, 256, 0, h->s>>>((const double*)src, dst, g, 0, g.nz + 1);
  else k_unpack<float><<<nb, 256, 0, h->s>>>((const float*)src, dst, g, 0, g.nz + 1);
  ++h->launches;
  CKL();
  return MG_OK;
}

// Galerkin level l: A_l = R A_{l-1} P in float64 from the level above (its
// 7-point edge coefficients or its 27-point couplings), then the V-cycle
// precision copies, D^-1 and the Gershgorin bound of D^-1 A_l.
mg_status build_galerkin_level(mg_handle* h, int l) {
  LevelBuf& Lv = h->lv[l];
  const LevelBuf& F = h->lv[l - 1];
  const i64 n = Lv.g.len;
  const size_t vb = vbytes(h), cb = cbytes(h);
  Lv.g27 = true;
  AL(Lv.w64, double, 13 * n);
  AL(Lv.dg64, double, n);
  FineOp fo{};
  fo.g = F.g;
  if (F.g27) {
    fo.w = F.w64;
    fo.dg = F.dg64;
    fo.wst = F.g.len;
  } else {
    fo.kx = F.kx64;
    fo.ky = F.ky64;
    fo.kz = F.kz64;
  }
  k_galerkin<<<lin_blocks(h, Lv.g.npts()), 128, 0, h->s>>>(fo, Lv.g, Lv.w64, Lv.dg64);
  CKL();
  void* q;
  AL(q, char, 13 * n * (i64)cb);
  Lv.w = q;
  AL(q, char, n * (i64)vb);
  Lv.dg = q;
  AL(q, char, n * (i64)vb);
  Lv.dinv = q;
  const int nb = lin_blocks(h, 13 * n);
  switch (h->prm.precision) {
    case MG_MIXED_FP32:
      k_cast<float, double><<<nb, 256, 0, h->s>>>(Lv.w64, (float*)Lv.w, 13 * n);
      k_diag27<float><<<lin_blocks(h, Lv.g.npts()), 256, 0, h->s>>>(Lv.dg64, (float*)Lv.dg, (float*)Lv.dinv, Lv.g);
      break;
    case MG_MIXED_BF16K:
      k_cast<__nv_bfloat16, double><<<nb, 256, 0, h->s>>>(Lv.w64, (__nv_bfloat16*)Lv.w, 13 * n);
      k_diag27<float><<<lin_blocks(h, Lv.g.npts()), 256, 0, h->s>>>(Lv.dg64, (float*)Lv.dg, (float*)Lv.dinv, Lv.g);
      break;
    default:
      k_cast<double, double><<<nb, 256, 0, h->s>>>(Lv.w64, (double*)Lv.w, 13 * n);
      k_diag27<double><<<lin_blocks(h, Lv.g.npts()), 256, 0, h->s>>>(Lv.dg64, (double*)Lv.dg, (double*)Lv.dinv,
                                                                       Lv.g);
  }
  CKL();
  CK(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned long long), h->s));
  k_gershgorin27<<<lin_blocks(h, Lv.g.npts()), 256, 0, h->s>>>(Lv.w64, Lv.dg64, Lv.g,
                                                               (unsigned long long*)h->dflag);
  CKL();
  double gb = 0.0;
  CK(cudaMemcpyAsync(&gb, h->dflag, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (!(gb > 0.0) || !std::isfinite(gb)) return fail(h, MG_ERR_NOT_SPD, "Galerkin coarse operator has a non-positive diagonal");
  Lv.beta = gb;
  return MG_OK;
}

// Level grids of the hierarchy (vertex counts per axis, level 0 finest), the
// level count and the first level of the bottom kernel, from the grid and the
// parameters alone (host arithmetic, no device).  Returns an error message,
// or an empty string.
std::string plan_hierarchy(int Nx, int Ny, int Nz, const mg_params& p, int N[MG_MAX_LEVELS][3], int* Lout,
                           int* lbout) {
  int L = p.levels;
  if (L <= 0) {
    L = 1;
    int M[3] = {Nx, Ny, Nz};
    while (L < MG_MAX_LEVELS) {
      bool ok = true;
      for (int a = 0; a < 3; ++a) ok = ok && (M[a] - 1) % 2 == 0 && (M[a] - 1) / 2 + 1 >= 5;
      if (!ok) break;
      for (int a = 0; a < 3; ++a) M[a] = (M[a] - 1) / 2 + 1;
      ++L;
    }
  }
  if (L > MG_MAX_LEVELS) return "too many levels";
  int M[3] = {Nx, Ny, Nz};
  for (int l = 0; l < L; ++l) {
    for (int a = 0; a < 3; ++a) {
      if (M[a] < 3) return "level grid has fewer than 3 vertices on an axis";
      N[l][a] = M[a];
    }
    if (l + 1 < L)
      for (int a = 0; a < 3; ++a) {
        if ((M[a] - 1) % 2) return "N-1 not divisible by 2^(levels-1)";
        M[a] = (M[a] - 1) / 2 + 1;
      }
  }
  auto npts = [&](int l) { return (i64)(N[l][0] - 2) * (N[l][1] - 2) * (N[l][2] - 2); };
  if (make_geom(N[0][0] - 2, N[0][1] - 2, N[0][2] - 2).len >= (i64)1 << 31)
    return "grid too large: padded arrays must stay below 2^31 elements";
  if (npts(L - 1) > MG_MAX_COARSE) return "coarsest level exceeds MG_MAX_COARSE unknowns";
  // telescoping: first level whose unknowns fit the bottom kernel
  int lb = L - 1;
  while (lb > 0 && npts(lb - 1) <= (i64)p.telescope_max_n && L - (lb - 1) <= BOT_MAX) --lb;
  *Lout = L;
  *lbout = lb;
  return std::string();
}

// z-slab partition (mg_params.slabs = S > 1): the agglomeration level la
// (slab_level, or the bottom kernel's first level, at most that) is split into
// S runs of consecutive interior planes, slab s owning planes
// [floor(s nz_la / S), floor((s+1) nz_la / S)); on every finer level l slab s
// owns the planes of its coarse planes, [a 2^(la-l), b 2^(la-l)), the last slab
// also the level's final plane (nz_l = 2 nz_{l+1} + 1).  So each slab's coarse
// planes restrict from its own fine planes plus the first fine plane of the
// next slab, and its fine planes prolongate from its own coarse planes plus
// the last coarse plane of the previous slab: one halo plane per neighbour.
// bounds[l*(S+1)+s] is slab s's first plane on level l, bounds[l*(S+1)+S] = nz_l.
std::string plan_slabs(int Nx, int Ny, int Nz, const mg_params& p, std::vector<int>* bounds, int* laout) {
  int N[MG_MAX_LEVELS][3], L = 0, lb = 0;
  std::string e = plan_hierarchy(Nx, Ny, Nz, p, N, &L, &lb);
  if (!e.empty()) return e;
  const int S = p.slabs;
  int la = p.slab_level > 0 ? p.slab_level : lb;
  if (la > lb) la = lb;
  if (la < 1) return "the slab decomposition needs at least one level above the agglomeration level";
  const int nz_la = N[la][2] - 2;
  if (S > nz_la) return "more slabs than interior planes on the agglomeration level";
  bounds->assign((size_t)(la + 1) * (S + 1), 0);
  for (int s = 0; s <= S; ++s) {
    const int a = (int)((long long)s * nz_la / S);
    for (int l = la; l >= 0; --l) (*bounds)[(size_t)l * (S + 1) + s] = s == S ? N[l][2] - 2 : a << (la - l);
  }
  *laout = la;
  return std::string();
}

mg_status build_hierarchy(mg_handle* h, int Nx, int Ny, int Nz, const double* k, int k_on_device) {
  const mg_params& p = h->prm;
  int N[MG_MAX_LEVELS][3];
  int L = 0;
  {
    const std::string e = plan_hierarchy(Nx, Ny, Nz, p, N, &L, &h->lb);
    if (!e.empty()) return fail(h, MG_ERR_ARG, e);
  }
  h->L = L;
  for (int l = 0; l < L; ++l) {
    LevelBuf& Lv = h->lv[l];
    for (int a = 0; a < 3; ++a) {
      Lv.N[a] = N[l][a];
      Lv.ih2[a] = (double)(N[l][a] - 1) * (double)(N[l][a] - 1);
    }
    Lv.g = make_geom(N[l][0] - 2, N[l][1] - 2, N[l][2] - 2);
  }
  const Geom& gc = h->lv[L - 1].g;
  h->nc = (int)gc.npts();
  // In float64 the bottom kernel's passes are bound by the float64 pipe of
  // its SM, and 27-point (Galerkin) passes by the work of one SM: a finest
  // bottom level of more than one point per thread then spreads over a
  // cluster of up to 8 blocks (8 SMs).  The float32 7-point passes are bound
  // by latency and barriers, which a cluster barrier does not improve
  // (measured on GB300 at 257^3: 7-point float32, one block is as fast as 4
  // or 8; 27-point float32, 4 blocks take the solve from 35.6 to 35.2 ms).
  {
    const i64 n0 = h->lv[h->lb].g.npts();
    int nb = 1;
    if (p.precision == MG_FP64 || (p.coarse_op == MG_COARSE_GALERKIN && h->lb >= 1))
      while (nb < 8 && n0 > (i64)nb * BOT_THREADS) nb *= 2;
    if (p.bottom_blocks > 0) nb = p.bottom_blocks;
    if (nb > 1 && !dispatch(h, [&](auto impl) { return decltype(impl)::bottom_cluster_fits(nb); })) nb = 1;
    h->bot_cluster = nb;
  }

  const bool mixed = p.precision != MG_FP64;
  const size_t vb = vbytes(h), cb = cbytes(h);
  // cells
  for (int l = 0; l < L; ++l) {
    LevelBuf& Lv = h->lv[l];
    const i64 ncell = (i64)(Lv.N[0] - 1) * (Lv.N[1] - 1) * (Lv.N[2] - 1);
    AL(Lv.kc, double, ncell);
    if (l == 0) {
      CK(cudaMemcpyAsync(Lv.kc, k, ncell * sizeof(double),
                         k_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
      CK(cudaMemsetAsync(h->dflag, 0, sizeof(int), h->s));
      k_cells_init<<<lin_blocks(h, ncell), 256, 0, h->s>>>(Lv.kc, ncell, p.k_is_log, h->dflag);
      CKL();
      int bad = 0;
      CK(cudaMemcpyAsync(&bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      if (bad) return fail(h, MG_ERR_NONFINITE, "k must be positive and finite in every cell");
    } else {
      const LevelBuf& F = h->lv[l - 1];
      k_coarsen_cells<<<lin_blocks(h, ncell), 256, 0, h->s>>>(F.kc, Lv.kc, Lv.N[0] - 1, Lv.N[1] - 1, Lv.N[2] - 1,
                                                              p.coarse_k_rule);
      CKL();
    }
  }
  // coefficients, diagonal and vectors per level
  for (int l = 0; l < L; ++l) {
    LevelBuf& Lv = h->lv[l];
    const i64 n = Lv.g.len;
    void* q;
    Lv.beta = p.eig_hi;
    if (l > 0 && p.coarse_op == MG_COARSE_GALERKIN) {
      mg_status sg = build_galerkin_level(h, l);
      if (sg != MG_OK) return sg;
    } else {
      for (void** c : {&Lv.kx, &Lv.ky, &Lv.kz}) {
        AL(q, char, n * (i64)cb);
        *c = q;
      }
      const bool need64 = !mixed || l == 0 || l == L - 1;
      if (mixed && need64) {
        AL(Lv.kx64, double, n);
        AL(Lv.ky64, double, n);
        AL(Lv.kz64, double, n);
      } else if (!mixed) {
        Lv.kx64 = (double*)Lv.kx;
        Lv.ky64 = (double*)Lv.ky;
        Lv.kz64 = (double*)Lv.kz;
      }
      const i64 nbox = (i64)(Lv.g.nx + 1) * (Lv.g.ny + 1) * (Lv.g.nz + 1);
      const int nb = lin_blocks(h, nbox);
      switch (p.precision) {
        case MG_MIXED_FP32:
          k_build_coef<float><<<nb, 256, 0, h->s>>>(Lv.kc, Lv.g, Lv.ih2[0], Lv.ih2[1], Lv.ih2[2], p.face_rule,
                                                    (float*)Lv.kx, (float*)Lv.ky, (float*)Lv.kz, Lv.kx64, Lv.ky64,
                                                    Lv.kz64);
          break;
        case MG_MIXED_BF16K:
          k_build_coef<__nv_bfloat16><<<nb, 256, 0, h->s>>>(
              Lv.kc, Lv.g, Lv.ih2[0], Lv.ih2[1], Lv.ih2[2], p.face_rule, (__nv_bfloat16*)Lv.kx,
              (__nv_bfloat16*)Lv.ky, (__nv_bfloat16*)Lv.kz, Lv.kx64, Lv.ky64, Lv.kz64);
          break;
        default:
          k_build_coef<double><<<nb, 256, 0, h->s>>>(Lv.kc, Lv.g, Lv.ih2[0], Lv.ih2[1], Lv.ih2[2], p.face_rule,
                                                     (double*)Lv.kx, (double*)Lv.ky, (double*)Lv.kz, nullptr,
                                                     nullptr, nullptr);
      }
      CKL();
      AL(q, char, n * (i64)vb);
      Lv.dinv = q;
      const int nbi = lin_blocks(h, Lv.g.npts());
      switch (p.precision) {
        case MG_MIXED_FP32:
          k_dinv<float, float, float><<<nbi, 256, 0, h->s>>>((float*)Lv.kx, (float*)Lv.ky, (float*)Lv.kz,
                                                             (float*)Lv.dinv, Lv.g);
          break;
        case MG_MIXED_BF16K:
          k_dinv<float, float, __nv_bfloat16><<<nbi, 256, 0, h->s>>>(
              (__nv_bfloat16*)Lv.kx, (__nv_bfloat16*)Lv.ky, (__nv_bfloat16*)Lv.kz, (float*)Lv.dinv, Lv.g);
          break;
        default:
          k_dinv<double, double, double><<<nbi, 256, 0, h->s>>>((double*)Lv.kx, (double*)Lv.ky, (double*)Lv.kz,
                                                                (double*)Lv.dinv, Lv.g);
      }
      CKL();
    }
    for (void** v : {&Lv.x[0], &Lv.x[1], &Lv.d, &Lv.r}) {
      AL(q, char, n * (i64)vb);
      *v = q;
    }
    if (l > 0 || mixed) {
      AL(q, char, n * (i64)vb);
      Lv.b = q;
    }
  }
  // outer CG vectors (float64, finest layout)
  const i64 n0 = h->lv[0].g.len;
  AL(h->cb, double, n0);
  AL(h->cx, double, n0);
  AL(h->cr, double, n0);
  AL(h->cq, double, n0);
  AL(h->cp, double, n0);
  AL(h->cw, double, n0);
  AL(h->dg64, double, n0);
  {
    const LevelBuf& L0 = h->lv[0];
    k_diag64<<<lin_blocks(h, L0.g.npts()), 256, 0, h->s>>>(L0.kx64, L0.ky64, L0.kz64, h->dg64, L0.g);
    CKL();
    if (p.test_inject == 1) {  // test only: an indefinite outer operator (p.Ap < 0)
      k_scale_strided<<<lin_blocks(h, n0), 256, 0, h->s>>>(h->dg64, -1.0, n0, 1);
      CKL();
    }
  }
  if (!mixed) h->lv[0].b = h->cr;  // the V-cycle's finest right-hand side is the CG residual
  // TMA-staged stencil kernels on the levels above the bottom kernel
  for (int l = 0; l < h->lb; ++l) {
    if (h->lv[l].g27) continue;  // the staged kernels read 7-point edge coefficients
    if (p.stencil_kernel == 1) {
      const bool ok = dispatch(h, [&](auto impl) { return decltype(impl)::tma_prepare(h, l); });
      if (!ok) return fail(h, MG_ERR_CUDA, "TMA tensor map encoding failed");
    }
  }
  CKL();
  // reduction scratch: enough for every reducing launch on the finest level
  int kcz;
  dim3 gz = zm_grid(h, h->lv[0].g, &kcz);
  // upper bound of the pointwise kernels' grids: every SM full of 256-thread blocks
  h->lin_grid = h->nsm * (2048 / LIN_THREADS);
  h->pstride = gz.x * gz.y * gz.z;
  {
    dim3 gv = zv_grid(h, h->lv[0].g, &kcz);
    const int vg = gv.x * gv.y * gv.z;
    if (h->pstride < vg) h->pstride = vg;
  }
  if (h->pstride < h->lin_grid) h->pstride = h->lin_grid;
  if (h->lv[0].tma) {
    const int tg = h->lv[0].tma_grid[0] * h->lv[0].tma_grid[1] * h->lv[0].tma_grid[2];
    if (h->pstride < tg) h->pstride = tg;
  }
  AL(h->partials, double, 2 * (i64)h->pstride);
  AL(h->dsc, Scal, 1);
  // Chebyshev intervals: the fixed (or Gershgorin) one, or the Lanczos estimate
  for (int l = 0; l < L; ++l) {
    LevelBuf& Lv = h->lv[l];
    if (p.eig_mode == 1) {
      double lm = 2.0;
      const mg_status se = dispatch(h, [&](auto impl) { return decltype(impl)::lanczos(h, l, &lm); });
      if (se != MG_OK) return se;
      if (!(lm > 0.0) || !std::isfinite(lm)) return fail(h, MG_ERR_NONFINITE, "eigenvalue estimate failed");
      Lv.beta = p.eig_safety * lm;
      Lv.alpha = p.eig_lo_frac * lm;
    } else {
      Lv.alpha = p.eig_lo_frac * Lv.beta;
    }
  }
  // coarsest operator: dense float64 assembly and Cholesky factorisation
  AL(h->Lc, double, (i64)h->nc * h->nc);
  const LevelBuf& Cv = h->lv[L - 1];
  if (Cv.g27) k_assemble_dense27<<<lin_blocks(h, h->nc), 256, 0, h->s>>>(Cv.w64, Cv.dg64, Cv.g, h->Lc);
  else k_assemble_dense<<<lin_blocks(h, h->nc), 256, 0, h->s>>>(Cv.kx64, Cv.ky64, Cv.kz64, Cv.g, h->Lc);
  CKL();
  if (p.coarse_solve == 1) {  // keep the operator for the inexact solve
    if (h->nc > 32) return fail(h, MG_ERR_ARG, "the inexact coarse solve needs at most 32 coarsest unknowns");
    AL(h->Ac, double, (i64)h->nc * h->nc);
    CK(cudaMemcpyAsync(h->Ac, h->Lc, sizeof(double) * h->nc * h->nc, cudaMemcpyDeviceToDevice, h->s));
  }
  if (p.test_inject == 2) {  // test only: a coarsest operator that is not positive definite
    k_scale_strided<<<1, 256, 0, h->s>>>(h->Lc, -1.0, (i64)h->nc, (i64)h->nc + 1);
    CKL();
  }
  CK(cudaMemsetAsync(h->dflag, 0, sizeof(int), h->s));
  k_cholesky<<<1, 1024, 0, h->s>>>(h->Lc, h->nc, h->dflag);
  CKL();
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (bad) return fail(h, MG_ERR_NOT_SPD, "coarsest operator is not positive definite");
  if (h->nc <= 32) {
    AL(h->Li, double, 2 * (i64)h->nc * h->nc);
    k_trinv<<<1, 32, 0, h->s>>>(h->Lc, h->Li, h->nc);
    CKL();
  }
  return MG_OK;
}

void release(mg_handle* h) {
  if (!h) return;
  if (h->sub) {  // a slab sub-hierarchy owns only its buffers
    for (void* p : h->allocs) cudaFree(p);
    delete h;
    return;
  }
  if (h->vexec) cudaGraphExecDestroy(h->vexec);
  if (h->s) cudaStreamSynchronize(h->s);
  for (mg_handle* c : h->slab) release(c);
  for (void* p : h->allocs) cudaFree(p);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  for (auto& pr : h->gap_ev)
    for (cudaEvent_t e : pr)
      if (e) cudaEventDestroy(e);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->ev_scal) cudaEventDestroy(h->ev_scal);
  if (h->s) cudaStreamDestroy(h->s);
  if (h->dflag) cudaFree(h->dflag);
  if (h->hsc) cudaFreeHost(h->hsc);
  if (h->khost) cudaFreeHost(h->khost);
  delete h;
}

// kernel classes launched inside the V-cycle (and its graph)
constexpr int VCYCLE_CLASSES = (1 << MG_K_CHEB_ZERO) | (1 << MG_K_CHEB_STEP) | (1 << MG_K_RESID) |
                               (1 << MG_K_RESTRICT) | (1 << MG_K_PROLONG) | (1 << MG_K_BOTTOM) | (1 << MG_K_DOT);

// Runs the V-cycle (and, in mixed precision, the casts around it); through a
// CUDA graph captured on first use when the handle enables graphs.

template <class I, class TV> mg_status run_precondition(mg_handle* h, TV** z) {
  NvtxRange range("mg V-cycle");
  if (!h->prm.use_graph || (h->timing && (h->t_cls_mask & VCYCLE_CLASSES))) {  // timed launches run eagerly
    *z = I::precondition(h);
    CKL();
    return MG_OK;
  }
  if (!h->vexec) {
    cudaGraph_t gr = nullptr;
    tm_collect(h);
    h->graph_recs.clear();
    h->ev_next = 0;
    CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    const long long before = h->launches;
    TV* zp = I::precondition(h);
    h->graph_launches = h->launches - before;
    h->launches = before;
    h->capturing = false;
    h->ev_graph_end = h->ev_next;
    cudaError_t e = cudaStreamEndCapture(h->s, &gr);
    if (e != cudaSuccess) return fail(h, MG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->vexec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      h->vexec = nullptr;
      return fail(h, MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    h->vexec_zcur = (zp == (TV*)h->lv[0].x[0]) ? 0 : 1;
  }
  CK(cudaGraphLaunch(h->vexec, h->s));
  h->launches += h->graph_launches;
  if (h->timing) h->pending.insert(h->pending.end(), h->graph_recs.begin(), h->graph_recs.end());
  *z = (TV*)h->lv[0].x[h->vexec_zcur];
  return MG_OK;
}

// Orders the internal stream after the caller's stream on entry and the
// caller's stream after the internal one on exit.
struct Guard {
  mg_handle* h;
  explicit Guard(mg_handle* hh) : h(hh) {
    if (h) {
      cudaEventRecord(h->ev_in, h->us);
      cudaStreamWaitEvent(h->s, h->ev_in, 0);
    }
  }
  ~Guard() {
    if (h) {
      cudaEventRecord(h->ev_out, h->s);
      cudaStreamWaitEvent(h->us, h->ev_out, 0);
    }
  }
};

template <class I, bool FLEX, class TV>
mg_status cg_iteration(mg_handle* h, TV* z, const Geom& g, const LevelBuf& L0) {
  NvtxRange range("mg CG iteration");
  // x += alpha_prev p, p = z + beta p;  q = A p, p.q -> alpha;  r -= alpha q, r.r (and r.z_old)
  linear<false>(h, g.len, LinPUpd<TV>{z, h->cp, h->cx, h->dsc, 0.0, 0.0}, MG_K_CG_DIR);
  int nb = zmarch<true>(h, g, OpApplyPQ{h->cp, h->cq, h->dg64, L0.kx64, L0.ky64, L0.kz64}, MG_K_CG_APPLY, 0);
  finish(h, nb, FIN_PQ);
  if (h->prm.precision == MG_FP64)
    nb = linear<true>(h, g.len, LinCgUpd<TV, FLEX, false>{h->cr, h->cq, z, nullptr, h->dsc, 0.0}, MG_K_CG_UPD);
  else
    nb = linear<true>(h, g.len, LinCgUpd<TV, FLEX, true>{h->cr, h->cq, z, (float*)L0.b, h->dsc, 0.0}, MG_K_CG_UPD);
  finish(h, nb, FIN_RR, h->sub ? nullptr : h->hsc_dev);  // the host reads the scalars after this one
  return MG_OK;
}

constexpr double QUEUE_MARGIN = 8.0;  // on the squared residual norm

template <class I> mg_status solve_impl(mg_handle* h, const double* f, double* x, double rtol, mg_stats* st) {
  NvtxRange range("mg CG solve");
  using TV = typename I::TVt;
  auto t0 = clk::now();
  const Geom& g = h->lv[0].g;
  const LevelBuf& L0 = h->lv[0];
  const mg_params& p = h->prm;
  h->hist.clear();
  const long long launches0 = h->launches;
  mg_status s;
  if ((s = pack_level(h, 0, f, h->cb, true)) != MG_OK) return s;
  CK(cudaMemsetAsync(h->cx, 0, (size_t)g.len * 8, h->s));
  CK(cudaMemsetAsync(h->cp, 0, (size_t)g.len * 8, h->s));
  CK(cudaMemsetAsync(h->dsc, 0, sizeof(Scal), h->s));
  int nb = linear<true>(h, g.len, LinDot<double>{h->cb, h->cb});
  finish(h, nb, FIN_BB);
  if (p.nonzero_guess) {
    if ((s = pack_level(h, 0, x, h->cx, true)) != MG_OK) return s;
    OpResidualD<double> res{h->cx, h->cb, h->cr, h->dg64, L0.kx64, L0.ky64, L0.kz64};
    nb = zmarch<true>(h, g, res);
    finish(h, nb, FIN_RR);
  } else {
    CK(cudaMemcpyAsync(h->cr, h->cb, (size_t)g.len * 8, cudaMemcpyDeviceToDevice, h->s));
  }
  if ((s = read_scal(h)) != MG_OK) return s;
  Scal sc = *h->hsc;
  mg_status result = MG_OK;
  int it = 0;
  const double bb = sc.bb;
  if (sc.status & 1) return fail(h, MG_ERR_NONFINITE, "non-finite value in f or x");
  const double tol2 = rtol * rtol * bb;
  double rr = sc.rr;
  if (bb > 0) h->hist.push_back(std::sqrt(rr / bb));
  if (bb > 0 && rr > tol2) {
    TV* z = nullptr;
    I::cast_rhs(h);
    if ((s = run_precondition<I>(h, &z)) != MG_OK) return s;
    const bool gap_on = h->timing && ((h->t_cls_mask >> MG_K_HOST_GAP) & 1) && h->gap_ev[0][0];
    int gap_prev = -1;  // event pair recorded in the previous iteration, read after the next host sync
    // The next V-cycle needs only the residual this iteration writes, so it is
    // queued behind the copy of the CG scalars before the host waits for
    // them: the host's convergence test then overlaps the device's work.  A
    // V-cycle queued after the last iteration is wasted (about 1% of a solve),
    // so queueing stops once the last residual reduction predicts a residual
    // within a factor QUEUE_MARGIN of the tolerance (CG's reduction varies
    // from one iteration to the next; the margin stops it a few iterations
    // before the end, each of which then waits for the host, about 10 us).
    double rr_prev = rr, ratio = 1.0;
    bool queued = false;  // the next V-cycle is already queued
    for (it = 1; it <= p.maxit; ++it) {
      if (p.flexible) cg_iteration<I, true>(h, z, g, L0);
      else cg_iteration<I, false>(h, z, g, L0);
      const int gp = it & 1;
      if (gap_on) CK(cudaEventRecord(h->gap_ev[gp][0], h->s));
      if ((s = read_scal_issue(h, true)) != MG_OK) return s;
      queued = it < p.maxit && rr_prev * ratio > QUEUE_MARGIN * tol2;
      int gap_now = -1;  // pair completed in this iteration, read in the next (after its wait)
      if (queued) {
        if (gap_on) {
          CK(cudaEventRecord(h->gap_ev[gp][1], h->s));
          gap_now = gp;
        }
        if ((s = run_precondition<I>(h, &z)) != MG_OK) return s;
      }
      if ((s = read_scal_wait(h)) != MG_OK) return s;
      if (gap_prev >= 0) {  // recorded in the previous iteration, so complete now
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->gap_ev[gap_prev][0], h->gap_ev[gap_prev][1]));
        h->t_ms[MG_K_HOST_GAP][0] += ms;
        h->t_n[MG_K_HOST_GAP][0] += 1;
      }
      gap_prev = gap_now;
      sc = *h->hsc;
      if (sc.status & ST_TIMEOUT) {  // checked first: the blocks that gave up left their outputs unwritten
        result = fail(h, MG_ERR_DEVICE_TIMEOUT,
                      "a bounded wait in a TMA-staged kernel gave up; the iterate is invalid");
        break;
      }
      if (sc.status & 1) {
        result = fail(h, MG_ERR_NONFINITE, "non-finite value during the iteration");
        break;
      }
      if (sc.status & 2) {
        result = fail(h, MG_ERR_BREAKDOWN, "CG breakdown: p.Ap <= 0");
        break;
      }
      rr = sc.rr;
      h->hist.push_back(std::sqrt(rr / bb));
      ratio = rr_prev > 0 ? rr / rr_prev : 1.0;
      rr_prev = rr;
      if (rr <= tol2) break;
      if (it == p.maxit) {
        result = fail(h, MG_ERR_NOT_CONVERGED, "maximum number of iterations reached");
        break;
      }
      if (!queued) {
        if (gap_on) {
          CK(cudaEventRecord(h->gap_ev[gp][1], h->s));
          gap_prev = gp;
        }
        if ((s = run_precondition<I>(h, &z)) != MG_OK) return s;
      }
    }
    if (it > p.maxit) it = p.maxit;
    // the last iteration's x += alpha p (deferred updates stop at exit)
    linear<false>(h, g.len, LinXUpd{h->cx, h->cp, h->dsc, 0.0}, MG_K_CG_DIR);
  }
  if ((s = unpack_level(h, 0, h->cx, x, true)) != MG_OK) return s;
  // true residual in float64
  OpResidualD<double> res{h->cx, h->cb, h->cq, h->dg64, L0.kx64, L0.ky64, L0.kz64};
  nb = zmarch<true>(h, g, res);
  finish(h, nb, FIN_TRUE);
  if ((s = read_scal(h)) != MG_OK) return s;
  h->st.iters = it;
  h->st.bnorm = std::sqrt(bb);
  h->st.rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  h->st.true_rel_resid = bb > 0 ? std::sqrt(h->hsc->true_rr / bb) : 0.0;
  h->st.solve_s = secs(t0);
  h->st.kernel_launches = h->launches - launches0;
  if (st) *st = h->st;
  return result;
}

// ---- z-slab decomposition ----------------------------------------------------
// The levels above the agglomeration level are split into z-slabs
// (plan_slabs).  Each slab is a sub-hierarchy with the layout of a level of
// its own (Geom with its plane count) whose two pad planes hold the
// neighbouring slabs' boundary planes instead of zeros wherever a neighbour
// exists: the halo that a rank of a distributed run receives into a local
// buffer.  The kernels are those of the single-domain solve, unchanged; what
// the decomposition adds is
//   - the halo exchange of a pass's operand before every stencil or transfer
//     pass (the operand's boundary planes copied into the neighbours' pad
//     planes);
//   - every reduction finished in two steps: each slab's block sums, then the
//     slabs' sums added in slab order (the all-reduce);
//   - the agglomeration: the agglomeration level's right-hand side gathered
//     from the slabs into the root hierarchy (the handle's own), the root's
//     V-cycle from there down (its bottom kernel), and the correction
//     scattered back with one halo plane on each side.
// All slabs live on the handle's device and stream: a single-GPU execution of
// the decomposed algorithm, in which each copy stands for a peer copy or a
// send/receive between ranks.  Setup builds the global hierarchy and copies
// each slab's planes of the level operators (with their halo planes) out of
// it.  A slab records the launches of one V-cycle and of one CG iteration
// once; the solve replays every recorded pass on all slabs in turn.

// Copies the planes of a slab out of a global level array: local planes
// -1 .. nz_local (the halo planes included) from global planes z0-1 .. z1,
// together with the pad slots just outside them that a 27-point stencil reads.
mg_status copy_slab_planes(mg_handle* h, void* dst, const Geom& gl, const void* src, const Geom& gg, int z0, size_t es) {
  const i64 lo_l = gl.Px - 1, lo_g = (i64)z0 * gg.sz + gg.Px - 1, n = gl.len - lo_l;
  CK(cudaMemcpyAsync((char*)dst + lo_l * es, (const char*)src + lo_g * es, (size_t)n * es, cudaMemcpyDeviceToDevice,
                     h->s));
  return MG_OK;
}

mg_status build_slabs(mg_handle* h) {
  const mg_params& p = h->prm;
  const int S = p.slabs;
  int la = 0;
  {
    const std::string e = plan_slabs(h->lv[0].N[0], h->lv[0].N[1], h->lv[0].N[2], p, &h->slab_z0, &la);
    if (!e.empty()) return fail(h, MG_ERR_ARG, e);
  }
  h->nslab = S;
  h->la = la;
  h->rank_mode = p.slab_rank >= 0;
  h->slab_first = h->rank_mode ? p.slab_rank : 0;
  AL(h->slots, double, 2 * (i64)S);
  const size_t vb = vbytes(h), cb = cbytes(h);
  const bool mixed = p.precision != MG_FP64;
  const int s_end = h->rank_mode ? h->slab_first + 1 : S;
  for (int s = h->slab_first; s < s_end; ++s) {
    mg_handle* c = new (std::nothrow) mg_handle();
    if (!c) return fail(h, MG_ERR_ALLOC, "host allocation failed");
    h->slab.push_back(c);
    c->sub = true;
    c->prm = p;
    c->s = h->s;
    c->us = h->us;
    c->nsm = h->nsm;
    c->dsc = h->dsc;
    c->hsc = h->hsc;
    c->dflag = h->dflag;
    c->L = la + 1;
    c->lb = la;
    c->zvec = h->zvec;
    c->lin_grid = h->lin_grid;
    for (int l = 0; l <= la; ++l) {
      const LevelBuf& G = h->lv[l];
      LevelBuf& Lv = c->lv[l];
      const int z0 = h->slab_z0[(size_t)l * (S + 1) + s], z1 = h->slab_z0[(size_t)l * (S + 1) + s + 1];
      for (int a = 0; a < 3; ++a) {
        Lv.N[a] = G.N[a];
        Lv.ih2[a] = G.ih2[a];
      }
      Lv.N[2] = z1 - z0 + 2;
      Lv.g = make_geom(G.g.nx, G.g.ny, z1 - z0);
      Lv.beta = G.beta;
      Lv.alpha = G.alpha;
      Lv.g27 = G.g27;
      const i64 n = Lv.g.len;
      void* q;
      mg_handle* hh = h;
      auto slab_copy = [&](void** dst, const void* src, size_t es, int count) -> mg_status {
        if (!src) return MG_OK;
        void* d = nullptr;
        mg_status st = alloc<char>(hh, (char**)&d, n * (i64)es * count);
        if (st != MG_OK) return st;
        for (int o = 0; o < count; ++o) {
          st = copy_slab_planes(hh, (char*)d + (size_t)o * n * es, Lv.g, (const char*)src + (size_t)o * G.g.len * es,
                                G.g, z0, es);
          if (st != MG_OK) return st;
        }
        *dst = d;
        return MG_OK;
      };
      mg_status st = MG_OK;
      if (l < la) {  // the operators of the slab's levels
        if (G.g27) {
          if ((st = slab_copy(&Lv.w, G.w, cb, 13)) != MG_OK) return st;
          if ((st = slab_copy(&Lv.dg, G.dg, vb, 1)) != MG_OK) return st;
        } else {
          if ((st = slab_copy(&Lv.kx, G.kx, cb, 1)) != MG_OK) return st;
          if ((st = slab_copy(&Lv.ky, G.ky, cb, 1)) != MG_OK) return st;
          if ((st = slab_copy(&Lv.kz, G.kz, cb, 1)) != MG_OK) return st;
          if (l == 0 && mixed) {
            void* t = nullptr;
            if ((st = slab_copy(&t, G.kx64, 8, 1)) != MG_OK) return st;
            Lv.kx64 = (double*)t;
            if ((st = slab_copy(&t, G.ky64, 8, 1)) != MG_OK) return st;
            Lv.ky64 = (double*)t;
            if ((st = slab_copy(&t, G.kz64, 8, 1)) != MG_OK) return st;
            Lv.kz64 = (double*)t;
          } else if (!mixed) {
            Lv.kx64 = (double*)Lv.kx;
            Lv.ky64 = (double*)Lv.ky;
            Lv.kz64 = (double*)Lv.kz;
          }
        }
        if ((st = slab_copy(&Lv.dinv, G.dinv, vb, 1)) != MG_OK) return st;
      }
      for (void** v : {&Lv.x[0], &Lv.x[1], &Lv.d, &Lv.r}) {
        st = alloc<char>(c, (char**)&q, n * (i64)vb);
        if (st != MG_OK) return fail(h, st, c->err);
        *v = q;
      }
      if (l > 0 || mixed) {
        st = alloc<char>(c, (char**)&q, n * (i64)vb);
        if (st != MG_OK) return fail(h, st, c->err);
        Lv.b = q;
      }
    }
    // the slab's float64 CG vectors and finest diagonal
    const Geom& g0 = c->lv[0].g;
    for (double** v : {&c->cb, &c->cx, &c->cr, &c->cq, &c->cp, &c->cw}) {
      mg_status st = alloc<double>(c, v, g0.len);
      if (st != MG_OK) return fail(h, st, c->err);
    }
    {
      void* t = nullptr;
      mg_handle* hh = h;
      mg_status st = alloc<char>(hh, (char**)&t, g0.len * 8);
      if (st != MG_OK) return st;
      if ((st = copy_slab_planes(hh, t, g0, h->dg64, h->lv[0].g, h->slab_z0[s], 8)) != MG_OK) return st;
      c->dg64 = (double*)t;
    }
    if (!mixed) c->lv[0].b = c->cr;
    // reduction scratch of the slab's largest reducing launch
    int kcz;
    dim3 gz = zm_grid(c, g0, &kcz);
    dim3 gv = zv_grid(c, g0, &kcz);
    c->pstride = std::max((int)(gz.x * gz.y * gz.z), std::max((int)(gv.x * gv.y * gv.z), c->lin_grid));
    {
      mg_status st = alloc<double>(c, &c->partials, 2 * (i64)c->pstride);
      if (st != MG_OK) return fail(h, st, c->err);
    }
    c->lin_lo = g0.off;
    c->lin_hi = g0.off + (i64)g0.nz * g0.sz;
  }
  CKL();
  return MG_OK;
}

// Before a pass: each pair of neighbouring slabs swaps the operand's boundary
// planes into each other's pad planes (a slab's last plane to the next slab's
// lower pad plane, the next slab's first plane to its upper pad plane).
mg_status slab_exchange(mg_handle* h, const std::vector<std::vector<Pass>>& R, size_t i) {
  if (h->rank_mode) {  // the one local slab swaps planes with the neighbouring ranks
    const Pass& a = R[0][i];
    const size_t es = (size_t)a.halo_bytes, pb = (size_t)a.halo_g.sz * es;
    char* A = (char*)a.halo;
    const Geom& ga = a.halo_g;
    const int r = h->slab_first;
    const int lo = r > 0, hi = r + 1 < h->nslab;
    if (lo) CK(cudaMemcpyAsync(h->tr.send_lo, A + (size_t)ga.off * es, pb, cudaMemcpyDeviceToDevice, h->s));
    if (hi)
      CK(cudaMemcpyAsync(h->tr.send_hi, A + (size_t)(ga.off + (i64)(ga.nz - 1) * ga.sz) * es, pb,
                         cudaMemcpyDeviceToDevice, h->s));
    CKL();
    if (h->tr.exchange(h->tr.ctx, (long long)pb, lo, hi, (void*)h->s) != 0)
      return fail(h, MG_ERR_CUDA, "slab transport: halo exchange failed");
    if (lo) CK(cudaMemcpyAsync(A + (size_t)(ga.off - ga.sz) * es, h->tr.recv_lo, pb, cudaMemcpyDeviceToDevice, h->s));
    if (hi)
      CK(cudaMemcpyAsync(A + (size_t)(ga.off + (i64)ga.nz * ga.sz) * es, h->tr.recv_hi, pb, cudaMemcpyDeviceToDevice,
                         h->s));
    return MG_OK;
  }
  for (int s = 0; s + 1 < h->nslab; ++s) {
    const Pass& a = R[s][i];
    const Pass& b = R[s + 1][i];
    const size_t es = (size_t)a.halo_bytes, pb = (size_t)a.halo_g.sz * es;
    char* A = (char*)a.halo;
    char* B = (char*)b.halo;
    const Geom &ga = a.halo_g, &gb = b.halo_g;
    CK(cudaMemcpyAsync(B + (size_t)(gb.off - gb.sz) * es, A + (size_t)(ga.off + (i64)(ga.nz - 1) * ga.sz) * es, pb,
                       cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(A + (size_t)(ga.off + (i64)ga.nz * ga.sz) * es, B + (size_t)gb.off * es, pb,
                       cudaMemcpyDeviceToDevice, h->s));
  }
  return MG_OK;
}

// A reduction finished across the slabs: each slab's block sums into its
// slot, then the slots added in slab order and the CG scalars updated.
mg_status slab_finish(mg_handle* h, const int* nbs, int mode) {
  const int S = h->nslab;
  if (h->rank_mode) {  // this rank's sums, summed over the ranks by the transport
    launch(h, k_finish_partial, dim3(1), dim3(FIN_THREADS), 0, (const double*)h->slab[0]->partials, nbs[0],
           h->slab[0]->pstride, h->tr.reduce_buf, 1);
    CKL();
    if (h->tr.allreduce(h->tr.ctx, 2, (void*)h->s) != 0) return fail(h, MG_ERR_CUDA, "slab transport: all-reduce failed");
    launch(h, k_combine, dim3(1), dim3(32), 0, (const double*)h->tr.reduce_buf, 1, mode, h->dsc, h->prm.flexible);
    h->launches += 2;
    return MG_OK;
  }
  for (int s = 0; s < S; ++s)
    launch(h, k_finish_partial, dim3(1), dim3(FIN_THREADS), 0, (const double*)h->slab[s]->partials, nbs[s],
           h->slab[s]->pstride, h->slots + s, S);
  launch(h, k_combine, dim3(1), dim3(32), 0, (const double*)h->slots, S, mode, h->dsc, h->prm.flexible);
  h->launches += S + 1;
  return MG_OK;
}

// Bytes of the agglomeration level's largest slab block (rank mode).
i64 slab_block_bytes(const mg_handle* h) {
  const int S = h->nslab;
  int mz = 0;
  for (int s = 0; s < S; ++s)
    mz = std::max(mz, h->slab_z0[(size_t)h->la * (S + 1) + s + 1] - h->slab_z0[(size_t)h->la * (S + 1) + s]);
  return (i64)mz * h->lv[h->la].g.sz * (i64)vbytes(h);
}

// The agglomeration level: gather the slabs' right-hand sides into the root
// level, run the root's V-cycle from it, scatter its correction (with one halo
// plane on each side) back to the slabs.
template <class I> mg_status slab_agglomerate(mg_handle* h, int la) {
  using TV = typename I::TVt;
  const int S = h->nslab;
  LevelBuf& R = h->lv[la];
  const i64 sz = R.g.sz;
  if (h->rank_mode) {  // every rank gathers all blocks and runs the whole-grid V-cycle itself
    const LevelBuf& C = h->slab[0]->lv[la];
    const i64 bb = slab_block_bytes(h);
    CK(cudaMemcpyAsync(h->tr.gather_send, (const TV*)C.b + C.g.off, (size_t)C.g.nz * sz * sizeof(TV),
                       cudaMemcpyDeviceToDevice, h->s));
    CKL();
    if (h->tr.allgather(h->tr.ctx, (long long)bb, (void*)h->s) != 0)
      return fail(h, MG_ERR_CUDA, "slab transport: all-gather failed");
    for (int q = 0; q < S; ++q) {
      const int z0 = h->slab_z0[(size_t)la * (S + 1) + q], z1 = h->slab_z0[(size_t)la * (S + 1) + q + 1];
      CK(cudaMemcpyAsync((TV*)R.b + R.g.off + (i64)z0 * sz, (const char*)h->tr.gather_recv + (size_t)q * bb,
                         (size_t)(z1 - z0) * sz * sizeof(TV), cudaMemcpyDeviceToDevice, h->s));
    }
    const int cur = I::vcycle(h, la);
    LevelBuf& M = h->slab[0]->lv[la];
    const int z0 = h->slab_z0[(size_t)la * (S + 1) + h->slab_first];
    CK(cudaMemcpyAsync((TV*)M.x[0] + M.g.off - sz, (const TV*)R.x[cur] + R.g.off + (i64)(z0 - 1) * sz,
                       (size_t)(M.g.nz + 2) * sz * sizeof(TV), cudaMemcpyDeviceToDevice, h->s));
    return MG_OK;
  }
  for (int s = 0; s < S; ++s) {
    const LevelBuf& C = h->slab[s]->lv[la];
    const int z0 = h->slab_z0[(size_t)la * (S + 1) + s];
    CK(cudaMemcpyAsync((TV*)R.b + R.g.off + (i64)z0 * sz, (const TV*)C.b + C.g.off, (size_t)C.g.nz * sz * sizeof(TV),
                       cudaMemcpyDeviceToDevice, h->s));
  }
  const int cur = I::vcycle(h, la);
  for (int s = 0; s < S; ++s) {
    LevelBuf& C = h->slab[s]->lv[la];
    const int z0 = h->slab_z0[(size_t)la * (S + 1) + s];
    CK(cudaMemcpyAsync((TV*)C.x[0] + C.g.off - sz, (const TV*)R.x[cur] + R.g.off + (i64)(z0 - 1) * sz,
                       (size_t)(C.g.nz + 2) * sz * sizeof(TV), cudaMemcpyDeviceToDevice, h->s));
  }
  return MG_OK;
}

// Replays a recorded phase on all slabs, pass by pass.
template <class I> mg_status slab_replay(mg_handle* h, const std::vector<std::vector<Pass>>& R) {
  const int S = (int)h->slab.size();  // the slabs this process holds
  std::vector<int> nbs(S);
  mg_status st;
  for (size_t i = 0; i < R[0].size(); ++i) {
    const Pass& p0 = R[0][i];
    switch (p0.kind) {
      case Pass::LAUNCH:
        if (p0.halo && (st = slab_exchange(h, R, i)) != MG_OK) return st;
        for (int s = 0; s < S; ++s) R[s][i].fn();
        h->launches += S;
        break;
      case Pass::MEMSET:
        for (int s = 0; s < S; ++s) R[s][i].fn();
        break;
      case Pass::FINISH:
        for (int s = 0; s < S; ++s) nbs[s] = R[s][i].nb;
        if ((st = slab_finish(h, nbs.data(), p0.mode)) != MG_OK) return st;
        break;
      case Pass::AGGLOM:
        if ((st = slab_agglomerate<I>(h, p0.level)) != MG_OK) return st;
        break;
    }
  }
  CKL();
  return MG_OK;
}

// Records one V-cycle and one CG iteration of every slab (once per handle).
template <class I, bool FLEX> mg_status slab_record(mg_handle* h) {
  using TV = typename I::TVt;
  if (!h->vrec.empty()) return MG_OK;
  const int S = (int)h->slab.size();
  h->vrec.assign(S, {});
  h->crec.assign(S, {});
  h->vz.assign(S, nullptr);
  for (int s = 0; s < S; ++s) {
    mg_handle* c = h->slab[s];
    c->rec = &h->vrec[s];
    TV* z = I::precondition(c);
    c->rec = &h->crec[s];
    cg_iteration<I, FLEX>(c, z, c->lv[0].g, c->lv[0]);
    c->rec = nullptr;
    h->vz[s] = z;
  }
  for (int s = 1; s < S; ++s) {  // every slab runs the same passes
    if (h->vrec[s].size() != h->vrec[0].size() || h->crec[s].size() != h->crec[0].size())
      return fail(h, MG_ERR_ARG, "slab sub-hierarchies recorded different pass sequences");
    for (size_t i = 0; i < h->vrec[0].size(); ++i)
      if (h->vrec[s][i].kind != h->vrec[0][i].kind) return fail(h, MG_ERR_ARG, "slab pass sequences differ");
  }
  return MG_OK;
}

// The decomposed CG solve: the steps of solve_impl with every vector split
// over the slabs.
template <class I> mg_status slab_solve(mg_handle* h, const double* f, double* x, double rtol, mg_stats* st) {
  NvtxRange range("mg z-slab CG solve");
  auto t0 = clk::now();
  const mg_params& p = h->prm;
  const int S = (int)h->slab.size();  // the slabs this process holds
  const int gs0 = h->slab_first;      // global index of the first of them
  const Geom& gG = h->lv[0].g;
  const i64 plane = (i64)(gG.nx + 2) * (gG.ny + 2);  // elements per dense full-grid plane
  h->hist.clear();
  const long long launches0 = h->launches;
  mg_status s;
  if (h->rank_mode && !h->tr_set) return fail(h, MG_ERR_ARG, "slab_rank >= 0 needs a transport (mg_set_transport)");
  if ((s = p.flexible ? slab_record<I, true>(h) : slab_record<I, false>(h)) != MG_OK) return s;
  std::vector<int> nbs(S);
  CK(cudaMemsetAsync(h->dsc, 0, sizeof(Scal), h->s));
  for (int q = 0; q < S; ++q) {
    mg_handle* c = h->slab[q];
    const Geom& g = c->lv[0].g;
    k_pack<double><<<lin_blocks(h, g.npts()), 256, 0, h->s>>>(f + (i64)h->slab_z0[gs0 + q] * plane, c->cb, g);
    CK(cudaMemsetAsync(c->cx, 0, (size_t)g.len * 8, h->s));
    CK(cudaMemsetAsync(c->cp, 0, (size_t)g.len * 8, h->s));
    CK(cudaMemcpyAsync(c->cr, c->cb, (size_t)g.len * 8, cudaMemcpyDeviceToDevice, h->s));
    nbs[q] = linear<true>(c, g.len, LinDot<double>{c->cb, c->cb});
  }
  if ((s = slab_finish(h, nbs.data(), FIN_BB)) != MG_OK) return s;
  if ((s = read_scal(h)) != MG_OK) return s;
  Scal sc = *h->hsc;
  mg_status result = MG_OK;
  int it = 0;
  const double bb = sc.bb;
  if (sc.status & 1) return fail(h, MG_ERR_NONFINITE, "non-finite value in f");
  const double tol2 = rtol * rtol * bb;
  double rr = sc.rr;
  if (bb > 0) h->hist.push_back(std::sqrt(rr / bb));
  if (bb > 0 && rr > tol2) {
    for (int q = 0; q < S; ++q) I::cast_rhs(h->slab[q]);
    if ((s = slab_replay<I>(h, h->vrec)) != MG_OK) return s;
    for (it = 1; it <= p.maxit; ++it) {
      if ((s = slab_replay<I>(h, h->crec)) != MG_OK) return s;
      if ((s = read_scal(h)) != MG_OK) return s;
      sc = *h->hsc;
      if (sc.status & 1) {
        result = fail(h, MG_ERR_NONFINITE, "non-finite value during the iteration");
        break;
      }
      if (sc.status & 2) {
        result = fail(h, MG_ERR_BREAKDOWN, "CG breakdown: p.Ap <= 0");
        break;
      }
      rr = sc.rr;
      h->hist.push_back(std::sqrt(rr / bb));
      if (rr <= tol2) break;
      if (it == p.maxit) {
        result = fail(h, MG_ERR_NOT_CONVERGED, "maximum number of iterations reached");
        break;
      }
      if ((s = slab_replay<I>(h, h->vrec)) != MG_OK) return s;
    }
    if (it > p.maxit) it = p.maxit;
    for (int q = 0; q < S; ++q) {
      mg_handle* c = h->slab[q];
      linear<false>(c, c->lv[0].g.len, LinXUpd{c->cx, c->cp, h->dsc, 0.0});
    }
  }
  // x: each slab writes its own planes (the first and last slab also the boundary planes)
  for (int q = 0; q < S; ++q) {
    mg_handle* c = h->slab[q];
    const Geom& g = c->lv[0].g;
    const int gq = gs0 + q;
    const int kf = gq == 0 ? 0 : 1, kl = gq == h->nslab - 1 ? g.nz + 1 : g.nz;
    k_unpack<double><<<lin_blocks(h, (i64)(g.nx + 2) * (g.ny + 2) * (kl - kf + 1)), 256, 0, h->s>>>(
        c->cx, x + (i64)h->slab_z0[gq] * plane, g, kf, kl);
  }
  // true residual in float64: halo exchange of x, residual and its norm per slab
  {
    std::vector<std::vector<Pass>> R(S, std::vector<Pass>(1));
    for (int q = 0; q < S; ++q) {
      R[q][0].halo = h->slab[q]->cx;
      R[q][0].halo_bytes = 8;
      R[q][0].halo_g = h->slab[q]->lv[0].g;
    }
    if ((s = slab_exchange(h, R, 0)) != MG_OK) return s;
    for (int q = 0; q < S; ++q) {
      mg_handle* c = h->slab[q];
      const LevelBuf& C0 = c->lv[0];
      OpResidual<double, double, double, double> res{c->cx, c->cb, c->cq, C0.kx64, C0.ky64, C0.kz64};
      nbs[q] = zmarch<true>(c, C0.g, res);
    }
    if ((s = slab_finish(h, nbs.data(), FIN_TRUE)) != MG_OK) return s;
  }
  if ((s = read_scal(h)) != MG_OK) return s;
  h->st.iters = it;
  h->st.bnorm = std::sqrt(bb);
  h->st.rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  h->st.true_rel_resid = bb > 0 ? std::sqrt(h->hsc->true_rr / bb) : 0.0;
  h->st.solve_s = secs(t0);
  for (mg_handle* c : h->slab) {
    h->launches += c->launches;
    c->launches = 0;
  }
  h->st.kernel_launches = h->launches - launches0;
  if (st) *st = h->st;
  return result;
}

// Flexible GMRES(m) preconditioned on the right by the V-cycle (Saad, Alg.
// 9.6), the outer Krylov method of the paper's Sec. 5 runs.  Classical
// Gram-Schmidt in float64 with the dot products of one column in one pass
// over the basis; Givens rotations and the small triangular solve on the
// host; restarts from the true residual every m steps.  Stops when the
// rotated residual norm |g_{j+1}| <= rtol ||b||.
mg_status fgmres_alloc(mg_handle* h) {
  if (h->kv) return MG_OK;
  const i64 n = h->lv[0].g.len;
  const int m = h->prm.gmres_restart;
  int per_sm = 0;  // one wave of the multi-dot kernel's resident blocks
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mdot<KR_MAXV>, KR_THREADS, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 2;
  }
  h->kgrid = h->nsm * per_sm;
  AL(h->kv, double, (i64)(m + 1) * n);
  void* q;
  AL(q, char, (i64)m * n * (i64)vbytes(h));
  h->kz = q;
  AL(h->kh, double, 2 * (i64)(m + 2));
  AL(h->kpart, double, std::max((i64)KR_MAXV * h->kgrid, (i64)lin_blocks(h, n)));  // k_mdot's and k_maxpy's partials
  if (cudaMallocHost(&h->khost, sizeof(double) * 2 * (m + 2)) != cudaSuccess) {
    cudaGetLastError();
    h->khost = nullptr;
    return fail(h, MG_ERR_ALLOC, "pinned host allocation failed");
  }
  return MG_OK;
}

// dst[v] = w . V_v for v < nv (V_v = V0 + v * n), in chunks of KR_MAXV vectors
void mdot(mg_handle* h, const double* w, const double* V0, int nv, double* dst) {
  const i64 n = h->lv[0].g.len;
  for (int c = 0; c < nv; c += KR_MAXV) {
    const int k = nv - c < KR_MAXV ? nv - c : KR_MAXV;
    const double* Vc = V0 + (i64)c * n;
    // chunks of 8, 4, 2 or 1 vectors (the kernel keeps 8 vectors' worth of loads in flight).
    // Grids measured on GB300 at 255^3: 2 blocks per SM for 8 and 4 vectors, 3 for 2 and 1.
    for (int d = 0; d < k;) {
      const int r = k - d, q = r >= 8 ? 8 : r >= 4 ? 4 : r >= 2 ? 2 : 1;
      const int grid = std::min(h->kgrid, h->nsm * (q >= 4 ? 2 : 3));
      switch (q) {
        case 8: k_mdot<8><<<grid, KR_THREADS, 0, h->s>>>(w, Vc + (i64)d * n, n, n, h->kpart); break;
        case 4: k_mdot<4><<<grid, KR_THREADS, 0, h->s>>>(w, Vc + (i64)d * n, n, n, h->kpart); break;
        case 2: k_mdot<2><<<grid, KR_THREADS, 0, h->s>>>(w, Vc + (i64)d * n, n, n, h->kpart); break;
        default: k_mdot<1><<<grid, KR_THREADS, 0, h->s>>>(w, Vc + (i64)d * n, n, n, h->kpart); break;
      }
      k_mdot_finish<<<q, KR_THREADS, 0, h->s>>>(h->kpart, grid, dst + c + d);
      h->launches += 2;
      d += q;
    }
  }
}

template <class I> mg_status fgmres_impl(mg_handle* h, const double* f, double* x, double rtol, mg_stats* st) {
  NvtxRange range("mg FGMRES solve");
  using TV = typename I::TVt;
  auto t0 = clk::now();
  const Geom& g = h->lv[0].g;
  const LevelBuf& L0 = h->lv[0];
  const mg_params& p = h->prm;
  const i64 n = g.len;
  const int m = p.gmres_restart;
  h->hist.clear();
  const long long launches0 = h->launches;
  mg_status s;
  if ((s = fgmres_alloc(h)) != MG_OK) return s;
  if ((s = pack_level(h, 0, f, h->cb, true)) != MG_OK) return s;
  if (p.nonzero_guess) {
    if ((s = pack_level(h, 0, x, h->cx, true)) != MG_OK) return s;
  } else {
    CK(cudaMemsetAsync(h->cx, 0, (size_t)n * 8, h->s));
  }
  CK(cudaMemsetAsync(h->dsc, 0, sizeof(Scal), h->s));
  int nb = linear<true>(h, n, LinDot<double>{h->cb, h->cb});
  finish(h, nb, FIN_BB);
  if ((s = read_scal(h)) != MG_OK) return s;
  const double bb = h->hsc->bb;
  if (!std::isfinite(bb)) return fail(h, MG_ERR_NONFINITE, "non-finite value in f");
  const double bnorm = std::sqrt(bb), tol = rtol * bnorm;
  const int lb = lin_blocks(h, n);
  double* V = h->kv;
  TV* Z = (TV*)h->kz;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1), y(m);
  mg_status result = MG_OK;
  int it = 0;
  double rnorm = 0.0;
  bool converged = false;
  while (bnorm > 0.0) {
    // restart from the true residual r = b - A x
    OpResidualD<double> res{h->cx, h->cb, h->cr, h->dg64, L0.kx64, L0.ky64, L0.kz64};
    nb = zmarch<true>(h, g, res);
    finish(h, nb, FIN_RR);
    if ((s = read_scal(h)) != MG_OK) return s;
    const double beta = std::sqrt(h->hsc->rr);
    if (!std::isfinite(beta)) {
      result = fail(h, MG_ERR_NONFINITE, "non-finite value in x or during the iteration");
      break;
    }
    rnorm = beta;
    if (h->hist.empty()) h->hist.push_back(beta / bnorm);
    if (beta <= tol) {
      converged = true;
      break;
    }
    if (it >= p.maxit) break;
    k_scale<<<lb, 256, 0, h->s>>>(V, h->cr, 1.0 / beta, n);
    ++h->launches;
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jj = 0;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      double* Vj = V + (i64)j * n;
      TV* Zj = Z + (i64)j * n;
      // z_j = M^-1 v_j: the V-cycle reads the float64 residual buffer (float64
      // form) or its float32 copy
      if (p.precision == MG_FP64) {
        CK(cudaMemcpyAsync(h->cr, Vj, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->s));
      } else {
        launch(h, k_cast<TV, double>, dim3(lb), dim3(256), 0, (const double*)Vj, (TV*)L0.b, n);
        ++h->launches;
      }
      TV* zp = nullptr;
      if ((s = run_precondition<I>(h, &zp)) != MG_OK) return s;
      CK(cudaMemcpyAsync(Zj, zp, (size_t)n * sizeof(TV), cudaMemcpyDeviceToDevice, h->s));
      // w = A z_j, then classical Gram-Schmidt against v_0..v_j
      zmarch<false>(h, g, OpApplyTo64<TV>{Zj, h->cw, h->dg64, L0.kx64, L0.ky64, L0.kz64});
      mdot(h, h->cw, V, j + 1, h->kh);
      // w -= V h, with the block sums of w.w of the updated w
      k_maxpy<double, true, true><<<lb, KR_THREADS, 0, h->s>>>(h->cw, V, n, j + 1, h->kh, n, h->kpart);
      k_mdot_finish<<<1, KR_THREADS, 0, h->s>>>(h->kpart, lb, h->kh + j + 1);
      h->launches += 2;
      CK(cudaMemcpyAsync(h->khost, h->kh, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      tm_collect(h);
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h->khost[i];
      const double hn = std::sqrt(h->khost[j + 1]);
      if (!std::isfinite(hn)) {
        result = fail(h, MG_ERR_NONFINITE, "non-finite value during the iteration");
        stop = true;
        break;
      }
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) {
        k_scale<<<lb, 256, 0, h->s>>>(V + (i64)(j + 1) * n, h->cw, 1.0 / hn, n);
        ++h->launches;
      }
      for (int i = 0; i < j; ++i) {  // earlier rotations on column j
        const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      const double d = std::sqrt(a * a + c * c);
      if (!(d > 0.0)) {
        result = fail(h, MG_ERR_BREAKDOWN, "GMRES breakdown: zero column");
        stop = true;
        break;
      }
      cs[j] = a / d;
      sn[j] = c / d;
      H[(size_t)j * m + j] = d;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++it;
      jj = j + 1;
      rnorm = std::fabs(gv[j + 1]);
      h->hist.push_back(rnorm / bnorm);
      if (rnorm <= tol || it >= p.maxit || hn == 0.0) {
        stop = true;
        break;
      }
    }
    // x += Z y with R y = g
    for (int i = jj - 1; i >= 0; --i) {
      double v = gv[i];
      for (int k = i + 1; k < jj; ++k) v -= H[(size_t)i * m + k] * y[k];
      y[i] = v / H[(size_t)i * m + i];
    }
    if (jj > 0) {
      for (int i = 0; i < jj; ++i) h->khost[i] = y[i];
      CK(cudaMemcpyAsync(h->kh, h->khost, sizeof(double) * jj, cudaMemcpyHostToDevice, h->s));
      k_maxpy<TV, false, false><<<lb, KR_THREADS, 0, h->s>>>(h->cx, Z, n, jj, h->kh, n, nullptr);
      ++h->launches;
      CK(cudaStreamSynchronize(h->s));  // the pinned y is reused by the next cycle
    }
    if (result != MG_OK) break;
    if (stop && rnorm <= tol) {
      converged = true;
      break;
    }
    if (stop && it >= p.maxit) break;
  }
  if (result == MG_OK && bnorm > 0.0 && !converged)
    result = fail(h, MG_ERR_NOT_CONVERGED, "maximum number of iterations reached");
  if ((s = unpack_level(h, 0, h->cx, x, true)) != MG_OK) return s;
  OpResidualD<double> res{h->cx, h->cb, h->cq, h->dg64, L0.kx64, L0.ky64, L0.kz64};
  nb = zmarch<true>(h, g, res);
  finish(h, nb, FIN_TRUE);
  if ((s = read_scal(h)) != MG_OK) return s;
  h->st.iters = it;
  h->st.bnorm = bnorm;
  h->st.rel_resid = bnorm > 0 ? rnorm / bnorm : 0.0;
  h->st.true_rel_resid = bnorm > 0 ? std::sqrt(h->hsc->true_rr / bb) : 0.0;
  h->st.solve_s = secs(t0);
  h->st.kernel_launches = h->launches - launches0;
  if (st) *st = h->st;
  return result;
}

}  // namespace

extern "C" {

mg_status mg_params_default(mg_params* p) {
  if (!p) return MG_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->levels = 0;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->cheby_degree = 2;
  p->eig_lo_frac = 0.1;
  p->eig_hi = 2.0;
  p->coarse_k_rule = 0;
  p->face_rule = 0;
  p->k_is_log = 0;
  p->precision = MG_FP64;
  p->maxit = 1000;
  p->nonzero_guess = 0;
  p->flexible = -1;
  p->telescope_max_n = 4096;
  p->use_graph = 1;
  p->stencil_kernel = 0;
  p->use_pdl = 1;
  p->smoother = MG_SMOOTHER_CHEBYSHEV;
  p->richardson_omega = 6.0 / 7.0;
  p->coarse_op = MG_COARSE_REDISCRETISED;
  p->krylov = MG_KRYLOV_CG;
  p->gmres_restart = 30;
  p->eig_mode = 0;
  p->eig_safety = 1.1;
  p->coarse_solve = 0;
  p->coarse_rtol = 1e-4;
  p->coarse_maxit = 30;
  p->bottom_blocks = 0;
  p->test_inject = 0;
  p->slabs = 1;
  p->slab_level = 0;
  p->slab_rank = -1;
  return MG_OK;
}

mg_status mg_setup(mg_handle** out, int Nx, int Ny, int Nz, const double* k_cells, int k_on_device,
                   const mg_params* prm, void* stream) {
  NvtxRange range("mg setup");
  auto t0 = clk::now();
  if (!out || !k_cells) return fail(nullptr, MG_ERR_ARG, "null handle or k pointer");
  *out = nullptr;
  mg_params p;
  if (prm) p = *prm;
  else mg_params_default(&p);
  if (Nx < 3 || Ny < 3 || Nz < 3) return fail(nullptr, MG_ERR_ARG, "grid needs at least 3 vertices per axis");
  if (p.nu_pre < 0 || p.nu_post < 0 || p.cheby_degree < 1 || p.cheby_degree > BOT_MAXDEG || p.maxit < 0 || !(p.eig_hi > 0) ||
      !(p.eig_lo_frac > 0 && p.eig_lo_frac < 1) || p.coarse_k_rule < 0 || p.coarse_k_rule > 2 || p.face_rule < 0 ||
      p.face_rule > 1 || p.precision < MG_FP64 || p.precision > MG_MIXED_BF16K || p.levels < 0 ||
      p.levels > MG_MAX_LEVELS || p.stencil_kernel < 0 || p.stencil_kernel > 2 ||
      p.smoother < MG_SMOOTHER_CHEBYSHEV || p.smoother > MG_SMOOTHER_RICHARDSON || !(p.richardson_omega > 0.0) ||
      p.coarse_op < MG_COARSE_REDISCRETISED || p.coarse_op > MG_COARSE_GALERKIN || p.krylov < MG_KRYLOV_CG ||
      p.krylov > MG_KRYLOV_FGMRES || p.gmres_restart < 1 || p.gmres_restart > 256 || p.eig_mode < 0 ||
      p.eig_mode > 1 || !(p.eig_safety > 0.0) || p.coarse_solve < 0 || p.coarse_solve > 1 ||
      !(p.coarse_rtol > 0.0) || p.coarse_maxit < 1 || p.coarse_maxit > 32 || (p.bottom_blocks != 0 && p.bottom_blocks != 1 && p.bottom_blocks != 2 && p.bottom_blocks != 4 && p.bottom_blocks != 8) ||
      p.test_inject < 0 || p.test_inject > 3 || p.slabs < 1 || p.slabs > MG_MAX_SLABS || p.slab_level < 0 || p.slab_rank < -1 ||
      p.slab_rank >= p.slabs || (p.slab_rank >= 0 && p.slabs < 2) ||
      (p.slabs > 1 && (p.krylov != MG_KRYLOV_CG || p.stencil_kernel == 1 || p.nonzero_guess)))
    return fail(nullptr, MG_ERR_ARG, "invalid mg_params");
  // Fletcher-Reeves by default: measured on GB300 the float32 / bfloat16
  // V-cycles need the same iteration counts with it as with the flexible
  // (Polak-Ribiere) beta, which costs one more dot product per iteration.
  if (p.flexible < 0) p.flexible = 0;
  // Richardson-Jacobi is the degree-1 Chebyshev step with theta = 1 / omega.
  if (p.smoother == MG_SMOOTHER_RICHARDSON) p.cheby_degree = 1;
  mg_handle* h = new (std::nothrow) mg_handle();
  if (!h) return fail(nullptr, MG_ERR_ALLOC, "host allocation failed");
  h->prm = p;
  h->zvec = p.stencil_kernel != 2;
  h->us = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (h->nsm <= 0) h->nsm = 152;
  mg_status s = MG_OK;
  if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_scal, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    s = fail(h, MG_ERR_CUDA, "stream or event creation failed");
  }
  if (s == MG_OK && (cudaMalloc(&h->dflag, sizeof(unsigned long long)) != cudaSuccess ||
                     cudaHostAlloc(&h->hsc, sizeof(Scal), cudaHostAllocMapped) != cudaSuccess ||
                     cudaHostGetDevicePointer((void**)&h->hsc_dev, h->hsc, 0) != cudaSuccess)) {
    cudaGetLastError();
    s = fail(h, MG_ERR_ALLOC, "scalar buffers");
  }
  Guard guard(s == MG_OK ? h : nullptr);
  if (s == MG_OK) s = build_hierarchy(h, Nx, Ny, Nz, k_cells, k_on_device);
  if (s == MG_OK && p.slabs > 1) s = build_slabs(h);
  if (s == MG_OK) s = sync_check(h);
  if (s != MG_OK) {
    g_setup_error = h->err;
    guard.h = nullptr;
    release(h);
    return s;
  }
  h->st.setup_s = secs(t0);
  *out = h;
  return MG_OK;
}

mg_status mg_set_stream(mg_handle* h, void* stream) {
  if (!h) return MG_ERR_ARG;
  h->us = (cudaStream_t)stream;
  return MG_OK;
}

mg_status mg_solve(mg_handle* h, const double* f, double* x, double rtol, mg_stats* st) {
  if (!h || !f || !x || !(rtol >= 0)) return h ? fail(h, MG_ERR_ARG, "null pointer or negative rtol") : MG_ERR_ARG;
  Guard guard(h);
  if (h->nslab > 1) return dispatch(h, [&](auto impl) { return slab_solve<decltype(impl)>(h, f, x, rtol, st); });
  if (h->prm.krylov == MG_KRYLOV_FGMRES)
    return dispatch(h, [&](auto impl) { return fgmres_impl<decltype(impl)>(h, f, x, rtol, st); });
  return dispatch(h, [&](auto impl) { return solve_impl<decltype(impl)>(h, f, x, rtol, st); });
}

mg_status mg_slab_transport_sizes(const mg_handle* h, long long* plane_bytes, long long* block_bytes) {
  if (!h || !plane_bytes || !block_bytes || !h->rank_mode) return MG_ERR_ARG;
  i64 pb = 0;
  for (int l = 0; l <= h->la; ++l)
    pb = std::max(pb, h->lv[l].g.sz * (i64)(l == 0 ? 8 : (i64)vbytes(h)));  // level 0 also exchanges float64 CG vectors
  *plane_bytes = pb;
  *block_bytes = slab_block_bytes(h);
  return MG_OK;
}

mg_status mg_set_transport(mg_handle* h, const mg_transport* t) {
  if (!h || !t || !h->rank_mode || !t->exchange || !t->allreduce || !t->allgather || !t->send_lo || !t->send_hi ||
      !t->recv_lo || !t->recv_hi || !t->reduce_buf || !t->gather_send || !t->gather_recv)
    return h ? fail(h, MG_ERR_ARG, "invalid transport (or the handle holds all slabs)") : MG_ERR_ARG;
  h->tr = *t;
  h->tr_set = true;
  return MG_OK;
}

mg_status mg_slab_plan(int Nx, int Ny, int Nz, const mg_params* p, int* bounds, int cap, int* agglomerate_level) {
  if (!p || !bounds || !agglomerate_level || p->slabs < 1 || p->slabs > MG_MAX_SLABS || p->slab_level < 0 ||
      p->telescope_max_n < 0)
    return fail(nullptr, MG_ERR_ARG, "invalid mg_slab_plan arguments");
  if (Nx < 3 || Ny < 3 || Nz < 3) return fail(nullptr, MG_ERR_ARG, "grid needs at least 3 vertices per axis");
  std::vector<int> b;
  int la = 0;
  const std::string e = plan_slabs(Nx, Ny, Nz, *p, &b, &la);
  if (!e.empty()) return fail(nullptr, MG_ERR_ARG, e);
  if ((int)b.size() > cap) return fail(nullptr, MG_ERR_ARG, "bounds array too small: (agglomeration level + 1) x (slabs + 1) entries");
  std::copy(b.begin(), b.end(), bounds);
  *agglomerate_level = la;
  return MG_OK;
}

mg_status mg_solve_host(mg_handle* h, const double* f_host, double* x_host, double rtol, mg_stats* st) {
  if (!h || !f_host || !x_host || !(rtol >= 0))
    return h ? fail(h, MG_ERR_ARG, "null pointer or negative rtol") : MG_ERR_ARG;
  auto t0 = clk::now();
  const LevelBuf& L0 = h->lv[0];
  const size_t bytes = sizeof(double) * (size_t)L0.N[0] * L0.N[1] * L0.N[2];
  Guard guard(h);
  if (!h->hstage[0]) {
    for (double*& b : h->hstage) AL(b, double, (i64)(bytes / sizeof(double)));
  }
  CK(cudaMemcpyAsync(h->hstage[0], f_host, bytes, cudaMemcpyHostToDevice, h->s));
  if (h->prm.nonzero_guess) CK(cudaMemcpyAsync(h->hstage[1], x_host, bytes, cudaMemcpyHostToDevice, h->s));
  mg_status s;
  if (h->nslab > 1)
    s = dispatch(h, [&](auto impl) { return slab_solve<decltype(impl)>(h, h->hstage[0], h->hstage[1], rtol, st); });
  else if (h->prm.krylov == MG_KRYLOV_FGMRES)
    s = dispatch(h, [&](auto impl) { return fgmres_impl<decltype(impl)>(h, h->hstage[0], h->hstage[1], rtol, st); });
  else
    s = dispatch(h, [&](auto impl) { return solve_impl<decltype(impl)>(h, h->hstage[0], h->hstage[1], rtol, st); });
  if (s != MG_OK && s != MG_ERR_NOT_CONVERGED && s != MG_ERR_BREAKDOWN && s != MG_ERR_NONFINITE &&
      s != MG_ERR_DEVICE_TIMEOUT)
    return s;
  CK(cudaMemcpyAsync(x_host, h->hstage[1], bytes, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  h->st.solve_s = secs(t0);  // the whole call, copies included
  if (st) *st = h->st;
  return s;
}

mg_status mg_gradient(mg_handle* h, const double* phi, const double* lambda, double* grad) {
  if (!h || !phi || !lambda || !grad) return h ? fail(h, MG_ERR_ARG, "null pointer") : MG_ERR_ARG;
  Guard guard(h);
  mg_status s;
  if ((s = pack_level(h, 0, phi, h->cw, true)) != MG_OK) return s;
  if ((s = pack_level(h, 0, lambda, h->cq, true)) != MG_OK) return s;
  const LevelBuf& L0 = h->lv[0];
  const i64 ncell = (i64)(L0.N[0] - 1) * (L0.N[1] - 1) * (L0.N[2] - 1);
  k_gradient<<<lin_blocks(h, ncell), 256, 0, h->s>>>(L0.kc, h->cw, h->cq, L0.g, L0.ih2[0],
                                                     L0.ih2[1], L0.ih2[2], h->prm.face_rule, grad);
  CKL();
  return MG_OK;
}

mg_status mg_solve_adjoint(mg_handle* h, const double* g, double* lambda, double rtol, const double* phi,
                           double* grad_logk, mg_stats* st) {
  if (!h || !g || !lambda || (grad_logk && !phi)) return h ? fail(h, MG_ERR_ARG, "null pointer") : MG_ERR_ARG;
  mg_status s = mg_solve(h, g, lambda, rtol, st);
  if (s != MG_OK) return s;
  if (grad_logk) {
    if ((s = mg_gradient(h, phi, lambda, grad_logk)) != MG_OK) return s;
    return sync_check(h);
  }
  return MG_OK;
}

mg_status mg_free(mg_handle* h) {
  if (!h) return MG_OK;
  cudaStreamSynchronize(h->s);
  release(h);
  return MG_OK;
}

const char* mg_last_error(const mg_handle* h) { return h ? h->err.c_str() : g_setup_error.c_str(); }

int mg_num_levels(const mg_handle* h) { return h ? h->L : 0; }

mg_status mg_level_dims(const mg_handle* h, int l, int* N3) {
  if (!h || !N3 || l < 0 || l >= h->L) return MG_ERR_ARG;
  for (int a = 0; a < 3; ++a) N3[a] = h->lv[l].N[a];
  return MG_OK;
}

mg_status mg_level_interval(const mg_handle* h, int l, double* alpha, double* beta) {
  if (!h || !alpha || !beta || l < 0 || l >= h->L) return MG_ERR_ARG;
  *alpha = h->lv[l].alpha;
  *beta = h->lv[l].beta;
  return MG_OK;
}

int mg_history(const mg_handle* h, double* hist, int cap) {
  if (!h) return 0;
  const int n = (int)h->hist.size();
  if (hist)
    for (int i = 0; i < n && i < cap; ++i) hist[i] = h->hist[i];
  return n;
}

mg_status mg_apply(mg_handle* h, int l, const double* x, double* y) {
  if (!h || !x || !y || l < -1 || l >= h->L) return h ? fail(h, MG_ERR_ARG, "bad level or pointer") : MG_ERR_ARG;
  Guard guard(h);
  mg_status s;
  if (l < 0) {
    const LevelBuf& L0 = h->lv[0];
    if ((s = pack_level(h, 0, x, h->cx, true)) != MG_OK) return s;
    OpApply<double, double, double> op{h->cx, h->cq, L0.kx64, L0.ky64, L0.kz64};
    zmarch<false>(h, L0.g, op);
    CKL();
    return unpack_level(h, 0, h->cq, y, true);
  }
  LevelBuf& Lv = h->lv[l];
  if ((s = pack_level(h, l, x, Lv.x[0], false)) != MG_OK) return s;
  dispatch(h, [&](auto impl) {
    using I = decltype(impl);
    using TV = std::remove_pointer_t<decltype(I::V(nullptr))>;
    using TC = std::remove_const_t<std::remove_pointer_t<decltype(I::C(nullptr))>>;
    if (Lv.g27) {
      OpApply27<TV, TV, TC> op{I::V(Lv.x[0]), I::V(Lv.r), I::C(Lv.w), Lv.g.len, I::V(Lv.dg)};
      zmarch<false>(h, Lv.g, op);
    } else {
      OpApply<TV, TV, TC> op{I::V(Lv.x[0]), I::V(Lv.r), I::C(Lv.kx), I::C(Lv.ky), I::C(Lv.kz)};
      zmarch<false>(h, Lv.g, op);
    }
    return 0;
  });
  CKL();
  return unpack_level(h, l, Lv.r, y, false);
}

mg_status mg_smooth(mg_handle* h, int l, const double* b, double* x, int zero_guess) {
  if (!h || !b || !x || l < 0 || l >= h->L) return h ? fail(h, MG_ERR_ARG, "bad level or pointer") : MG_ERR_ARG;
  Guard guard(h);
  LevelBuf& Lv = h->lv[l];
  mg_status s;
  if ((s = pack_level(h, l, b, Lv.b, false)) != MG_OK) return s;
  if (!zero_guess && (s = pack_level(h, l, x, Lv.x[0], false)) != MG_OK) return s;
  const int cur = dispatch(h, [&](auto impl) { return decltype(impl)::sweep(h, l, 0, zero_guess != 0); });
  CKL();
  return unpack_level(h, l, Lv.x[cur], x, false);
}

mg_status mg_residual_restrict(mg_handle* h, int l, const double* b, const double* x, double* bc) {
  if (!h || !b || !x || !bc || l < 0 || l + 1 >= h->L)
    return h ? fail(h, MG_ERR_ARG, "bad level or pointer") : MG_ERR_ARG;
  Guard guard(h);
  LevelBuf& Lv = h->lv[l];
  LevelBuf& Cv = h->lv[l + 1];
  mg_status s;
  if ((s = pack_level(h, l, b, Lv.b, false)) != MG_OK) return s;
  if ((s = pack_level(h, l, x, Lv.x[0], false)) != MG_OK) return s;
  dispatch(h, [&](auto impl) {
    decltype(impl)::residual_restrict(h, l, 0);
    return 0;
  });
  CKL();
  return unpack_level(h, l + 1, Cv.b, bc, false);
}

mg_status mg_prolong_add(mg_handle* h, int l, const double* ec, double* x) {
  if (!h || !ec || !x || l < 0 || l + 1 >= h->L) return h ? fail(h, MG_ERR_ARG, "bad level or pointer") : MG_ERR_ARG;
  Guard guard(h);
  LevelBuf& Lv = h->lv[l];
  LevelBuf& Cv = h->lv[l + 1];
  mg_status s;
  if ((s = pack_level(h, l + 1, ec, Cv.x[0], false)) != MG_OK) return s;
  if ((s = pack_level(h, l, x, Lv.x[0], false)) != MG_OK) return s;
  dispatch(h, [&](auto impl) {
    using I = decltype(impl);
    using TV = std::remove_pointer_t<decltype(I::V(nullptr))>;
    OpProlong<TV, TV> pr{Cv.g, I::V(Cv.x[0]), I::V(Lv.x[0])};
    zmarch<false>(h, Lv.g, pr);
    return 0;
  });
  CKL();
  return unpack_level(h, l, Lv.x[0], x, false);
}

mg_status mg_coarse_solve(mg_handle* h, const double* b, double* x) {
  if (!h || !b || !x) return h ? fail(h, MG_ERR_ARG, "null pointer") : MG_ERR_ARG;
  Guard guard(h);
  const int l = h->L - 1;
  LevelBuf& Lv = h->lv[l];
  mg_status s;
  if ((s = pack_level(h, l, b, Lv.b, false)) != MG_OK) return s;
  dispatch(h, [&](auto impl) {
    decltype(impl)::bottom(h, l);
    return 0;
  });
  CKL();
  return unpack_level(h, l, Lv.x[0], x, false);
}

mg_status mg_vcycle(mg_handle* h, const double* r, double* z) {
  if (!h || !r || !z) return h ? fail(h, MG_ERR_ARG, "null pointer") : MG_ERR_ARG;
  Guard guard(h);
  mg_status s;
  if ((s = pack_level(h, 0, r, h->cr, true)) != MG_OK) return s;
  void* zp = dispatch(h, [&](auto impl) {
    decltype(impl)::cast_rhs(h);
    return (void*)decltype(impl)::precondition(h);
  });
  CKL();
  return unpack_level(h, 0, zp, z, false);
}

mg_status mg_residual_norm(mg_handle* h, const double* f, const double* x, double* out) {
  if (!h || !f || !x || !out) return h ? fail(h, MG_ERR_ARG, "null pointer") : MG_ERR_ARG;
  Guard guard(h);
  const LevelBuf& L0 = h->lv[0];
  mg_status s;
  if ((s = pack_level(h, 0, f, h->cb, true)) != MG_OK) return s;
  if ((s = pack_level(h, 0, x, h->cx, true)) != MG_OK) return s;
  OpResidualD<double> res{h->cx, h->cb, h->cq, h->dg64, L0.kx64, L0.ky64, L0.kz64};
  const int nb = zmarch<true>(h, L0.g, res);
  finish(h, nb, FIN_TRUE);
  if ((s = read_scal(h)) != MG_OK) return s;
  *out = std::sqrt(h->hsc->true_rr);
  return MG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Residual norm for callers that cannot allocate: per-plane partial sums live
// in this file-scope device array instead of the handle's scratch buffers.
namespace {

static __device__ __align__(256) double g_noalloc_partials[MG_NOALLOC_MAX_PLANES];

constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mutex;

// Device address of g_noalloc_partials on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// One block per interior plane k: sum over the plane of (f - A x)^2 with f and
// x in the dense full-grid layout (boundary entries treated as zero) and the
// float64 operator read from the handle's padded coefficient arrays.
__global__ void __launch_bounds__(256) k_resnorm_planes(const double* __restrict__ f, const double* __restrict__ x,
                                                        const double* __restrict__ kx, const double* __restrict__ ky,
                                                        const double* __restrict__ kz, const double* __restrict__ dg,
                                                        Geom g, double* partials) {
  const int k = blockIdx.x;
  const int Nx = g.nx + 2, Ny = g.ny + 2, Nz = g.nz + 2;
  const i64 sy = Nx, sz = (i64)Nx * Ny;
  auto X = [&](int I, int J, int K) -> double {
    const bool in = I >= 1 && I <= Nx - 2 && J >= 1 && J <= Ny - 2 && K >= 1 && K <= Nz - 2;
    return in ? x[(i64)K * sz + (i64)J * sy + I] : 0.0;
  };
  double acc = 0.0, unused = 0.0;
  const int n = g.nx * g.ny;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % g.nx, j = t / g.nx;
    const int I = i + 1, J = j + 1, K = k + 1;
    const i64 p = g.at(i, j, k);
    const double S = kx[p - 1] * X(I - 1, J, K) + kx[p] * X(I + 1, J, K) + ky[p - g.Px] * X(I, J - 1, K) +
                     ky[p] * X(I, J + 1, K) + kz[p - g.sz] * X(I, J, K - 1) + kz[p] * X(I, J, K + 1);
    const double r = f[(i64)K * sz + (i64)J * sy + I] - (dg[p] * X(I, J, K) - S);
    acc = fma(r, r, acc);
  }
  block_sum2<256>(acc, unused);
  if (threadIdx.x == 0) partials[k] = acc;
}

// Sum of the per-plane partials in plane order; out = sqrt(sum).
__global__ void __launch_bounds__(256) k_resnorm_sum(const double* partials, int n, double* out) {
  double a = 0.0, unused = 0.0;
  for (int t = threadIdx.x; t < n; t += 256) a += partials[t];
  block_sum2<256>(a, unused);
  if (threadIdx.x == 0) out[0] = sqrt(a);
}

}  // namespace

extern "C" {

mg_status mg_residual_norm_noalloc(mg_handle* h, const double* f, const double* x, double* out) {
  if (!h || !f || !x || !out) return h ? fail(h, MG_ERR_ARG, "null pointer") : MG_ERR_ARG;
  const LevelBuf& L0 = h->lv[0];
  if (L0.g.nz > MG_NOALLOC_MAX_PLANES)
    return fail(h, MG_ERR_ARG, "mg_residual_norm_noalloc: grid has more than MG_NOALLOC_MAX_PLANES interior planes");
  double* scratch = nullptr;
  CK(noalloc_scratch(&scratch));
  Guard guard(h);
  k_resnorm_planes<<<L0.g.nz, 256, 0, h->s>>>(f, x, L0.kx64, L0.ky64, L0.kz64, h->dg64, L0.g, scratch);
  k_resnorm_sum<<<1, 256, 0, h->s>>>(scratch, L0.g.nz, out);
  CKL();
  return MG_OK;
}

mg_status mg_timing_enable(mg_handle* h, int class_mask, int level_mask) {
  const int on = class_mask != 0;
  if (!h) return MG_ERR_ARG;
  CK(cudaStreamSynchronize(h->s));
  if (on && h->evpool.empty()) {
    h->evpool.resize(EV_POOL);
    for (auto& e : h->evpool) CK(cudaEventCreate(&e));
    for (auto& pr : h->gap_ev)
      for (cudaEvent_t& e : pr) CK(cudaEventCreate(&e));
  }
  if (h->vexec) {
    cudaGraphExecDestroy(h->vexec);
    h->vexec = nullptr;
  }
  h->timing = on;
  h->t_cls_mask = class_mask;
  h->t_lvl_mask = level_mask;
  h->graph_recs.clear();
  h->pending.clear();
  h->ev_graph_end = h->ev_next = 0;
  std::memset(h->t_ms, 0, sizeof(h->t_ms));
  std::memset(h->t_n, 0, sizeof(h->t_n));
  std::memset(h->t_pts, 0, sizeof(h->t_pts));
  return MG_OK;
}

mg_status mg_timing_read(const mg_handle* h, int cls, int l, double* ms, long long* launches, double* points) {
  if (!h || cls < 0 || cls >= MG_K_NCLASS || l < 0 || l >= MG_MAX_LEVELS) return MG_ERR_ARG;
  if (ms) *ms = h->t_ms[cls][l];
  if (launches) *launches = h->t_n[cls][l];
  if (points) *points = h->t_pts[cls][l];
  return MG_OK;
}

}  // extern "C"
