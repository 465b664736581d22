// libamr4 orchestration and C-ABI entry points: composite operators (COH-1..4), the
// composite V-cycle (Sec. 6.5), solves with the max-norm stopping test (Sec. 7), the
// solvability fix (Sec. 6.4), the composite projection (Eq. comp_ProjOp) and FP32 V-cycles
// inside FP64 iterative refinement.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "amr4_impl.h"
#include "kernels.cuh"
#include "sweep3d.cuh"
#include "coarse3d.cuh"
#include "cic.cuh"
#include "migrate.cuh"

using namespace amr4;

namespace {

// ---------------------------------------------------------------- scratch and operator
template <typename T>
struct Scratch {
  T* E = nullptr;   // per-level corrections
  T* R = nullptr;   // per-level right-hand sides / residuals
  T* T1 = nullptr;  // smoothing ping-pong
  T* T2 = nullptr;
  T* X = nullptr;   // accumulated composite correction
  T* rin = nullptr; // V-cycle input residual (FP32 path)
  T* Z = nullptr;   // composite transpose: masked input
  T* W = nullptr;   // composite transpose: accumulated result
  T* Y = nullptr;   // adjoint V-cycle temporary
  std::vector<T*> mx, mb, mt;  // level-0 multigrid grids m >= 1
  bool ready = false;
};

}  // namespace

struct amr_operator {
  amr_hierarchy* h = nullptr;
  double alpha = 0.0, beta = 1.0;
  int bc[6] = {0, 0, 0, 0, 0, 0};
  bool neumann = false;  // pure-Neumann PPE: alpha == 0 and every face Neumann
  double* d_binv = nullptr;
  double* d_binvT = nullptr;  // transposed inverse (adjoint V-cycles)
  int nbot = 0, ldb = 0;
  Scratch<double> s64;
  Scratch<float> s32;
  double* F = nullptr;    // internal right-hand side copy
  double* Res = nullptr;  // FP64 composite residual
  double* Tmp = nullptr;  // FP64 composite scratch
  std::vector<XferBlock*> d_mgx;  // transfer block m -> m+1
  double* hphi = nullptr;  // device staging for the host-buffer solve (allocated once)
  double* hf = nullptr;
  double* hbc = nullptr;
  // captured solve (use_graph): one graph = prologue + device-side while loop over V-cycles
  struct DevStats* d_stats = nullptr;   // one per replica of a stacked component batch
  struct DevStats* h_stats = nullptr;   // pinned
  int* d_active = nullptr;              // replicas still iterating (stacked batches)
  unsigned long long* h_cnorm = nullptr;  // pinned copy of the per-replica norms
  struct StackCtx* stack = nullptr;       // stacked batch led by this operator (amr_batch_solve)
  double* h_scal = nullptr;            // pinned copy of the hierarchy's device scalars
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* g_phi = nullptr;
  const void* g_bc = nullptr;
  int g_prec = -1, g_nu1 = -1, g_nu2 = -1, g_maxv = -1;
  double g_omega = 0.0, g_rtol = -1.0, g_atol = -1.0;
  long long launches_pre = 0, launches_body = 0;
  int g_fuse = -1;
  int g_blk = -1;
  int g_cpr = 1;                  // cycles per refinement step of the captured solve
  float* inner_x = nullptr;       // mixed precision, cycles_per_refinement > 1: the correction so far
  float* inner_r = nullptr;       // and the FP32 composite residual of the correction equation
  int cmg_m0[2][2] = {{-1, -1}, {-1, -1}};  // [transpose][precision 0 = FP32, 1 = FP64]; -1: unset
  size_t cmg_bytes[2][2] = {{0, 0}, {0, 0}};
};

struct DevStats {
  int iter;    // V-cycles performed
  int status;  // 0 converged, 1 max_vcycles reached, 2 non-finite residual, 3 running
  double hist[64];
};

namespace {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
      return AMR_ERR_CUDA;                                                            \
    }                                                                                 \
  } while (0)

#define TRY(...)                         \
  do {                                   \
    amr_status s_ = (__VA_ARGS__);       \
    if (s_ != AMR_OK) return s_;         \
  } while (0)

std::atomic<long long> g_launches{0};  // kernels launched by this library (host count)

thread_local cudaError_t g_launch_err = cudaSuccess;

// Launch with programmatic stream serialisation (see pdl_wait): the next kernel's launch and
// block scheduling overlap the tail of the current one, inside captured graphs as well.
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess && g_launch_err == cudaSuccess) g_launch_err = e;
}

inline amr_status launch_check() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && g_launch_err != cudaSuccess) e = g_launch_err;
  g_launch_err = cudaSuccess;
  if (e != cudaSuccess) {
    set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return AMR_ERR_CUDA;
  }
  return AMR_OK;
}

// Bulk-copy 3-D sweep (k_sweep3d) on single-patch levels whose x extent is a multiple of 64
// and y extent a multiple of the tile height.  amr_set_bulk_sweep: 0 never, 1 (default) where
// the tile autotuner finds it fastest, 2 wherever eligible.
std::atomic<int> g_bulk_sweep{1};
std::atomic<int> g_stack_batches{0};  // amr_set_stacked_batches
#ifndef SW_TILE_Y
#define SW_TILE_Y 16
#endif
#ifndef SW_ROWS_PER_WARP
#define SW_ROWS_PER_WARP 2
#endif
#ifndef SW_STAGES
#define SW_STAGES 8
#endif
constexpr int SW_TY = SW_TILE_Y, SW_RW = SW_ROWS_PER_WARP, SW_S = SW_STAGES, SW_MINZ = 8;
inline bool sw_eligible(const LevelView& lv) {
  if (g_bulk_sweep.load(std::memory_order_relaxed) == 0 || lv.D != 3 || lv.npatch != lv.ncomp) return false;
  if (lv.maxn[0] % sw3::TX != 0 || lv.maxn[1] % SW_TY != 0 || lv.maxn[2] < 4) return false;
  const long long px = ((lv.maxn[0] + 2 * NG) + 3) / 4 * 4;
  return px * (lv.maxn[1] + 2 * NG) * (lv.maxn[2] + 2 * NG) < (1LL << 31);
}
constexpr int TILE_BULK = 8;  // tile-table code of the bulk-copy 3-D kernel

void free_stack(amr_operator* op);  // stacked component batches (defined with amr_batch_solve)

// ---------------------------------------------------------------- tile autotuner
// Rows per thread of the tiled 2-D kernel and of the z-chunked 3-D kernel, per (dimension,
// grid cells, value size): filled by autotune_tiles() (CUDA-event timing of each variant on
// the operator's own buffers), with a size-based default before tuning.
std::mutex g_tile_mu;
std::vector<std::pair<long long, int>> g_tile_table;

inline long long tile_key(const LevelView& lv, size_t tsize) {
  return ((long long)lv.ncells * 4 + lv.D) * 16 + (long long)tsize;
}

std::atomic<int> g_tile_force{0};  // amr_set_tile_rows: 0 = autotuned

inline int tile_rows_for(const LevelView& lv, size_t tsize) {
  const int forced = g_tile_force.load(std::memory_order_relaxed);
  if (forced) return lv.D == 3 ? std::max(2, forced) : forced;
  if (lv.D == 3 && g_bulk_sweep.load(std::memory_order_relaxed) == 2 && sw_eligible(lv)) return TILE_BULK;
  const long long key = tile_key(lv, tsize);
  {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    for (const auto& e : g_tile_table)
      if (e.first == key) return e.second;
  }
  if (lv.D == 3) {
    const int mode = g_bulk_sweep.load(std::memory_order_relaxed);
    return (sw_eligible(lv) && (mode == 2 || lv.ncells >= 2097152.0)) ? TILE_BULK : 2;
  }
  return lv.ncells >= 1024.0 * 1024.0 ? 4 : 1;
}

template <typename T>
inline T pick_host(double d, float f);
template <>
inline double pick_host<double>(double d, float) { return d; }
template <>
inline float pick_host<float>(double, float f) { return f; }

// ---------------------------------------------------------------- bench instrumentation
// When enabled, launches of the instrumented kernel classes are bracketed with CUDA events
// on the launching stream; amr_profile_read() sums the event intervals.
enum { PC_JACOBI = 0, PC_RESID = 1, PC_RESTRICT = 2, PC_PROLONG = 3, PC_DOWN = 4, PC_UP = 5, PC_COARSE = 6, PC_RESID64 = 7,
       PC_NCLASS = 8 };
struct ProfRec {
  cudaEvent_t a, b;
  int cls;
  double bytes;
  double cells;  // cells of the grid the launch worked on (0: not recorded)
};
struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
};
Profiler g_prof;
constexpr size_t PROF_MAX = 400000;

inline void prof_begin(cudaStream_t st, cudaEvent_t* ev) {
  if (!g_prof.on || g_prof.used + 2 > 2 * PROF_MAX) { *ev = nullptr; return; }
  *ev = g_prof.get();
  cudaEventRecord(*ev, st);
}
inline void prof_end(cudaStream_t st, cudaEvent_t a, int cls, double bytes, double cells = 0.0) {
  if (a == nullptr) return;
  cudaEvent_t b = g_prof.get();
  cudaEventRecord(b, st);
  g_prof.recs.push_back({a, b, cls, bytes, cells});
}

template <typename T>
amr_status dalloc(T** p, size_t n) {
  if (cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation failed");
    return AMR_ERR_OOM;
  }
  return AMR_OK;
}

struct Geo {
  dim3 grid;
  dim3 block{BX, BY, 1};
  int nby;
};

inline Geo geo_of(const LevelView& v) {
  Geo g;
  g.nby = (v.maxn[1] + BY - 1) / BY;
  g.grid = dim3((v.maxn[0] + BX - 1) / BX, g.nby * (v.D == 3 ? v.maxn[2] : 1), v.npatch);
  return g;
}

LevelView mg_view(const amr_hierarchy* h, int m, const int* bc) {
  LevelView v{};
  const MgGrid& g = h->mg[m];
  v.patches = g.d_patch;
  v.npatch = 1;
  v.D = h->D;
  v.h = g.h;
  for (int e = 0; e < 3; ++e) { v.ndom[e] = g.n[e]; v.maxn[e] = g.n[e]; }
  for (int f = 0; f < 6; ++f) { v.bc[f] = bc[f]; v.bc_off[f] = 0; v.bc_pitch[f] = 1; }
  v.ncells = (double)g.n[0] * g.n[1] * g.n[2] * h->ncomp;
  v.p0 = g.patch;
  v.npatch = h->ncomp;
  v.ncomp = h->ncomp;
  v.cstride = g.cstride;
  v.active = h->ncomp > 1 ? h->d_active : nullptr;
  finish_view(v);
  return v;
}

// range [first, end) of a level's elements inside a composite field
inline void level_range(const amr_hierarchy* h, int l, long long& a, long long& b, int comp = 0) {
  // replica comp of a stacked component batch: its patches are comp * (level's patches per
  // replica) onwards, its layout ends at (comp + 1) * cstride
  const int npl = (int)h->lev[l].patches.size() / h->ncomp;
  a = h->lev[l].patches[(size_t)comp * npl].off;
  if (l + 1 < h->L) {
    const int npn = (int)h->lev[l + 1].patches.size() / h->ncomp;
    b = h->lev[l + 1].patches[(size_t)comp * npn].off;
  } else {
    b = h->ncomp > 1 ? (comp + 1) * h->cstride : h->nelems;
  }
}

// ---------------------------------------------------------------- host bottom matrix
const double HG[2][2][4] = {{{-77.0 / 12.0, 43.0 / 12.0, -17.0 / 12.0, 3.0 / 12.0},
                              {-505.0 / 12.0, 335.0 / 12.0, -145.0 / 12.0, 27.0 / 12.0}},
                             {{5.0 / 10.0, 9.0 / 10.0, -5.0 / 10.0, 1.0 / 10.0},
                              {-75.0 / 10.0, 145.0 / 10.0, -75.0 / 10.0, 15.0 / 10.0}}};

// alpha x + beta L x on one box grid with homogeneous physical ghosts (host, for the
// dense bottom-solve matrix).
void host_apply(int D, const int n[3], double h, double alpha, double beta, const int* bc,
                const std::vector<double>& x, std::vector<double>& y) {
  auto at = [&](int i, int j, int k) -> double { return x[((size_t)k * n[1] + j) * n[0] + i]; };
  auto val = [&](int c0, int c1, int c2, int d) -> double {
    int c[3] = {c0, c1, c2};
    if (c[d] >= 0 && c[d] < n[d]) return at(c[0], c[1], c[2]);
    const int side = c[d] < 0 ? 0 : 1;
    const int layer = side == 0 ? -c[d] : c[d] - n[d] + 1;
    const int type = bc[2 * d + side];
    double v = 0.0;
    for (int m = 0; m < 4; ++m) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[d] = side == 0 ? m : n[d] - 1 - m;
      v += HG[type][layer - 1][m] * at(cc[0], cc[1], cc[2]);
    }
    return v;
  };
  y.assign(x.size(), 0.0);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        double acc = 0.0;
        int c[3] = {i, j, k};
        for (int d = 0; d < D; ++d) {
          int cm1[3] = {i, j, k}, cp1[3] = {i, j, k}, cm2[3] = {i, j, k}, cp2[3] = {i, j, k};
          cm1[d] = c[d] - 1; cp1[d] = c[d] + 1; cm2[d] = c[d] - 2; cp2[d] = c[d] + 2;
          acc += 16.0 * (val(cm1[0], cm1[1], cm1[2], d) + val(cp1[0], cp1[1], cp1[2], d)) -
                 (val(cm2[0], cm2[1], cm2[2], d) + val(cp2[0], cp2[1], cp2[2], d));
        }
        acc -= 30.0 * D * at(i, j, k);
        y[((size_t)k * n[1] + j) * n[0] + i] = alpha * at(i, j, k) + beta * acc / (12.0 * h * h);
      }
}

bool invert(std::vector<double>& A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = i;
    if (A[(size_t)piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
        std::swap(I[(size_t)c * n + k], I[(size_t)piv * n + k]);
      }
    const double d = A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) { A[(size_t)c * n + k] /= d; I[(size_t)c * n + k] /= d; }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = A[(size_t)i * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)i * n + k] -= f * A[(size_t)c * n + k];
        I[(size_t)i * n + k] -= f * I[(size_t)c * n + k];
      }
    }
  }
  A.swap(I);
  return true;
}

// ---------------------------------------------------------------- kernel wrappers
// The z-chunked 3-D operator runs on single-patch levels whose x / y extents are multiples of
// its 32 x 8R tile and whose padded patch has fewer than 2^31 elements (32-bit offsets).
inline bool zc_eligible(const LevelView& lv, int R) {
  // one patch per component (stacked component batches: ncomp replicas of one patch)
  if (lv.D != 3 || lv.npatch != lv.ncomp || lv.maxn[0] % ZC_TX != 0 || lv.maxn[1] % (ZC_TY * R) != 0 || lv.maxn[2] < MIN_BOX)
    return false;
  const long long px = ((lv.maxn[0] + 2 * NG) + 3) / 4 * 4;
  return px * (lv.maxn[1] + 2 * NG) * (lv.maxn[2] + 2 * NG) < (1LL << 31);
}

// One full wave of a kernel on the current device: resident blocks per SM (for the given
// block size and dynamic shared memory) times the device's SM count, queried once per
// (device, kernel) pair.
int wave_blocks(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, kernel});
  if (it != cache.end()) return it->second;
  int nsm = 0, per = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  const int blocks = std::max(1, std::max(1, nsm) * std::max(1, per));
  cache[{dev, kernel}] = blocks;
  return blocks;
}

// one full wave of the z-chunked 3-D kernel
template <typename T, int M, int R>
int zc_blocks() {
  return wave_blocks(reinterpret_cast<const void*>(k_level_op3d_zc<T, M, R>), ZC_TX * ZC_TY, 0);
}

// z chunks of the 3-D kernel: as many as one wave holds, at least 4 planes each
template <typename T, int M, int R>
void launch_zc(const LevelView& lv, const T* x, const T* f, T* out, T A, T B, T O, const unsigned char* vmask,
               cudaStream_t st, const unsigned* gate = nullptr) {
  const int ntx = lv.maxn[0] / ZC_TX, ntiles = ntx * (lv.maxn[1] / (ZC_TY * R)), nz = lv.maxn[2];
  const int nc = std::max(1, lv.ncomp);  // stacked component batches: one part of the grid per replica
  const int nch = std::max(1, std::min(zc_blocks<T, M, R>() / (ntiles * nc), nz / 4));
  const int kc = (nz + nch - 1) / nch;
  const int G = ntiles * ((nz + kc - 1) / kc);
  launch(k_level_op3d_zc<T, M, R>, G * nc, dim3(ZC_TX, ZC_TY, 1), 0, st, lv, ntx, ntiles, kc, x, f, out, A, B, O,
         vmask, gate);
}

template <typename T, int M>
constexpr auto sw_kernel() {
  return k_sweep3d<T, M, SW_TY, SW_RW, SW_S>;
}
template <typename T>
amr_status sw_attrs() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return AMR_OK;
  CK(cudaFuncSetAttribute(sw_kernel<T, OP_APPLY>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sw3::smem_bytes<T, OP_APPLY, SW_TY, SW_S>()));
  CK(cudaFuncSetAttribute(sw_kernel<T, OP_RESID>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sw3::smem_bytes<T, OP_RESID, SW_TY, SW_S>()));
  CK(cudaFuncSetAttribute(sw_kernel<T, OP_JACOBI>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sw3::smem_bytes<T, OP_JACOBI, SW_TY, SW_S>()));
  CK(cudaFuncSetAttribute(sw_kernel<T, OP_JACOBI0>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sw3::smem_bytes<T, OP_JACOBI0, SW_TY, SW_S>()));
  CK(cudaFuncSetAttribute(sw_kernel<T, OP_RESTRICT>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)sw3::smem_bytes<T, OP_RESTRICT, SW_TY, SW_S>()));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return AMR_OK;
}
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
using TmapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmapEncodeFn tmap_encoder() {
  static std::once_flag once;
  static TmapEncodeFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmapEncodeFn>(p);
  });
  return fn;
}

// Tensor map of a single-patch field over its padded patch (dimensions: row pitch, n_y + 4,
// n_z + 4), boxes of 68 x rows x 1 values.
template <typename T>
amr_status encode_patch_tmap(CUtensorMap* tm, const T* field, const PatchDesc& p, int rows, int ncomp,
                             long long cstride) {
  const TmapEncodeFn enc = tmap_encoder();
  if (enc == nullptr) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return AMR_ERR_CUDA;
  }
  // dimension 3: the replicas of a stacked component batch (extent 1 otherwise)
  const long long pz = p.n[2] + 2 * NG;
  const cuuint64_t dims[4] = {(cuuint64_t)p.sy, (cuuint64_t)(p.n[1] + 2 * NG), (cuuint64_t)pz,
                              (cuuint64_t)std::max(1, ncomp)};
  const cuuint64_t strides[3] = {(cuuint64_t)p.sy * sizeof(T), (cuuint64_t)p.sz * sizeof(T),
                                 (cuuint64_t)(ncomp > 1 ? cstride : p.sz * pz) * sizeof(T)};
  const cuuint32_t box[4] = {(cuuint32_t)sw3::XW, (cuuint32_t)rows, 1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r =
      enc(tm, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
          const_cast<T*>(field + p.off), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return AMR_ERR_CUDA;
  }
  return AMR_OK;
}

// tiles of 64 x SW_TY cells; z chunks of at least SW_MINZ planes, as many as one wave holds
template <typename T, int M>
amr_status launch_sw(const LevelView& lv, const T* x, const T* f, T* out, T A, T B, T O, const unsigned char* vmask,
                     cudaStream_t st, const unsigned* gate = nullptr, T* outc = nullptr, const PatchDesc* cpd = nullptr,
                     long long ccs = 0) {
  TRY(sw_attrs<T>());
  constexpr size_t smem = sw3::smem_bytes<T, M, SW_TY, SW_S>();
  constexpr int threads = 32 * (SW_TY / SW_RW + 2);
  CUtensorMap tmx{}, tmf{};
  const int nc = std::max(1, lv.ncomp);  // stacked component batches: one part of the grid per replica
  if (M != OP_JACOBI0) TRY(encode_patch_tmap<T>(&tmx, x, lv.p0, SW_TY + 4, nc, lv.cstride));
  if (M == OP_JACOBI0) TRY(encode_patch_tmap<T>(&tmf, f, lv.p0, SW_TY, nc, lv.cstride));
  const int ntx = lv.maxn[0] / sw3::TX, ntiles = ntx * (lv.maxn[1] / SW_TY), nz = lv.maxn[2];
  const int wave = wave_blocks(reinterpret_cast<const void*>(sw_kernel<T, M>()), threads, smem);
  const int nch = std::max(1, std::min(wave / (ntiles * nc), nz / SW_MINZ));
  launch(sw_kernel<T, M>(), (unsigned)(ntiles * nch * nc), threads, smem, st, tmx, tmf, lv, ntx, ntiles, nch, f, out,
         A, B, O, vmask, gate, outc, cpd != nullptr ? *cpd : PatchDesc{}, ccs);
  return launch_check();
}

// Clears and reports the flag that k_sweep3d sets when one of its bounded waits ran out.
amr_status sweep3d_check_flag() {
  unsigned v = 0u;
  CK(cudaMemcpyFromSymbol(&v, g_sweep3d_err, sizeof(unsigned)));
  if (v != 0u) {
    const unsigned z = 0u;
    CK(cudaMemcpyToSymbol(g_sweep3d_err, &z, sizeof(unsigned)));
    set_error("a bounded pipeline wait of the 3-D sweep kernel ran out (results of that solve are invalid)");
    return AMR_ERR_CUDA;
  }
  return AMR_OK;
}

// FP64 residual of a z-chunked level with the fixed-point stencil sums (k_resid3d_fx): the
// frame from the level's largest interior |x|, the fixed-point pass, and the plain FP64
// pass gated on the out-of-frame flag (it exits at once unless a value left the frame)
std::atomic<int> g_fx_resid{1};  // amr_set_fx_residual
inline bool fx_eligible(const LevelView& lv) {
  return lv.fxs != nullptr && g_fx_resid.load(std::memory_order_relaxed) != 0 && zc_eligible(lv, 2);
}
int fx_blocks() { return wave_blocks(reinterpret_cast<const void*>(k_resid3d_fx), ZC_TX * ZC_TY, 0); }
// the bulk-copy form (k_resid3d_fx_tma): tiles of 64 x SW_TY cells, two consumer rows per warp,
// four converter warps (of the shapes measured on 256^3, the fastest: 259 us per residual
// against 263 us with four rows and three converters, 280 us with two rows and three
// converters, 304 us with four rows and two converters)
#ifndef RFX_ROWS_PER_WARP
#define RFX_ROWS_PER_WARP 2
#endif
#ifndef RFX_CONVERTER_WARPS
#define RFX_CONVERTER_WARPS 4
#endif
constexpr int RFX_RW = RFX_ROWS_PER_WARP, RFX_NFW = RFX_CONVERTER_WARPS;
constexpr auto rfx_kernel() { return k_resid3d_fx_tma<SW_TY, RFX_RW, SW_S, RFX_NFW>; }
amr_status rfx_attrs() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return AMR_OK;
  CK(cudaFuncSetAttribute(rfx_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)rfx_smem_bytes<SW_TY, SW_S>()));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return AMR_OK;
}
amr_status launch_resid_fx(const LevelView& lv, const double* x, const double* f, double* out, double alpha,
                           double beta, cudaStream_t st) {
  const int nc = std::max(1, lv.ncomp);  // stacked component batches: a frame and a flag per replica
  CK(cudaMemsetAsync(lv.fxs, 0, 2 * nc * sizeof(unsigned long long), st));
  const long long rows = (long long)lv.maxn[1] * lv.maxn[2];
  const int amax_blocks = wave_blocks(reinterpret_cast<const void*>(k_absmax_patch), 256, 0);
  launch(k_absmax_patch, dim3((unsigned)std::min<long long>((rows + 7) / 8, std::max(1, amax_blocks / nc)), nc, 1), 256,
         0, st, lv, x, lv.fxs);
  TRY(launch_check());
  // the bulk-copy form where the bulk-copy sweep is forced, or on grids of 2^21 cells and
  // more (measured: 256^3 FP64 residual 259 us against 273 us; 128^3: 57 against 52 us)
  const int bulk = g_bulk_sweep.load(std::memory_order_relaxed);
  if (sw_eligible(lv) && (bulk == 2 || lv.ncells >= 2097152.0)) {
    TRY(rfx_attrs());
    constexpr size_t smem = rfx_smem_bytes<SW_TY, SW_S>();
    constexpr int threads = rfx_threads<SW_TY, RFX_RW, SW_S, RFX_NFW>();
    CUtensorMap tmx{}, tmf{};
    TRY(encode_patch_tmap<double>(&tmx, x, lv.p0, SW_TY + 4, nc, lv.cstride));
    TRY(encode_patch_tmap<double>(&tmf, f, lv.p0, SW_TY, nc, lv.cstride));
    const int ntx = lv.maxn[0] / sw3::TX, ntiles = ntx * (lv.maxn[1] / SW_TY), nz = lv.maxn[2];
    const int wave = wave_blocks(reinterpret_cast<const void*>(rfx_kernel()), threads, smem);
    const int nch = std::max(1, std::min(wave / (ntiles * nc), nz / SW_MINZ));
    launch(rfx_kernel(), (unsigned)(ntiles * nch * nc), threads, smem, st, tmx, tmf, lv, ntx, ntiles, nch, x, f,
           out, alpha, beta);
  } else {
    const int ntx = lv.maxn[0] / ZC_TX, ntiles = ntx * (lv.maxn[1] / (ZC_TY * 2)), nz = lv.maxn[2];
    const int nch = std::max(1, std::min(fx_blocks() / (ntiles * nc), nz / 4));
    const int kc = (nz + nch - 1) / nch;
    const int G = ntiles * ((nz + kc - 1) / kc);
    launch(k_resid3d_fx, G * nc, dim3(ZC_TX, ZC_TY, 1), 0, st, lv, ntx, ntiles, kc, x, f, out, alpha, beta);
  }
  TRY(launch_check());
  launch_zc<double, OP_RESID, 2>(lv, x, f, out, alpha, beta, 0.0, nullptr, st,
                                 reinterpret_cast<const unsigned*>(lv.fxs + 1));
  return launch_check();
}

template <typename T, int D, bool TR = false>
amr_status level_op(int mode, const LevelView& lv, const T* x, const T* f, T* out, const T* bc, double alpha,
                    double beta, double omega, const unsigned char* vmask, cudaStream_t st) {
  Geo g = geo_of(lv);
  cudaEvent_t ev;
  prof_begin(st, &ev);
  if (D == 2) {
    // tiled 2-D path; omega / (interior diagonal) computed once here in the value type;
    // rows per thread from the autotuner's table (keyed by grid size), default by size
    const T diag = T(alpha) + T(beta) * pick_host<T>(lv.inv12h2, lv.inv12h2_f) * T(-60);
    const T ood = T(omega) / diag;
    const int rows = tile_rows_for(lv, sizeof(T));
    dim3 grid((lv.maxn[0] + BX - 1) / BX, (lv.maxn[1] + BY * rows - 1) / (BY * rows), lv.npatch);
    dim3 block(BX, BY, 1);
    const T A = T(alpha), B = T(beta), O = T(omega);
#define LAUNCH_TILED(M)                                                                                     \
  do {                                                                                                      \
    if (rows == 4) launch(k_level_op2d_tiled<T, M, TR, 4>, grid, block, 0, st, lv, x, f, out, bc, A, B, O, ood, vmask); \
    else if (rows == 2) launch(k_level_op2d_tiled<T, M, TR, 2>, grid, block, 0, st, lv, x, f, out, bc, A, B, O, ood, vmask); \
    else launch(k_level_op2d_tiled<T, M, TR, 1>, grid, block, 0, st, lv, x, f, out, bc, A, B, O, ood, vmask); \
  } while (0)
    switch (mode) {
      case OP_APPLY: LAUNCH_TILED(OP_APPLY); break;
      case OP_RESID: LAUNCH_TILED(OP_RESID); break;
      case OP_JACOBI: LAUNCH_TILED(OP_JACOBI); break;
      default: LAUNCH_TILED(OP_JACOBI0);
    }
#undef LAUNCH_TILED
    const double nb = mode == OP_JACOBI0 ? 2.0 : (mode == OP_APPLY ? 2.0 : 3.0);
    prof_end(st, ev, (mode == OP_JACOBI || mode == OP_JACOBI0) ? PC_JACOBI : (mode == OP_RESID && sizeof(T) == 8) ? PC_RESID64 : PC_RESID,
             nb * sizeof(T) * lv.ncells, lv.ncells);
    return launch_check();
  }
  if constexpr (sizeof(T) == 8 && D == 3 && !TR) {
    if (mode == OP_RESID && bc == nullptr && vmask == nullptr && fx_eligible(lv)) {
      if (const amr_status s1 = launch_resid_fx(lv, x, f, out, alpha, beta, st); s1 != AMR_OK) return s1;
      prof_end(st, ev, PC_RESID64, 3.0 * sizeof(T) * lv.ncells, lv.ncells);
      return launch_check();
    }
  }
  if (D == 3 && !TR && bc == nullptr && (vmask == nullptr || mode == OP_RESID) && sw_eligible(lv) &&
      tile_rows_for(lv, sizeof(T)) == TILE_BULK) {
    const T A = T(alpha), B = T(beta), O = T(omega);
    amr_status s1;
    switch (mode) {
      case OP_APPLY: s1 = launch_sw<T, OP_APPLY>(lv, x, f, out, A, B, O, vmask, st); break;
      case OP_RESID: s1 = launch_sw<T, OP_RESID>(lv, x, f, out, A, B, O, vmask, st); break;
      case OP_JACOBI: s1 = launch_sw<T, OP_JACOBI>(lv, x, f, out, A, B, O, vmask, st); break;
      default: s1 = launch_sw<T, OP_JACOBI0>(lv, x, f, out, A, B, O, vmask, st);
    }
    if (s1 != AMR_OK) return s1;
    const double nb = mode == OP_JACOBI0 ? 2.0 : (mode == OP_APPLY ? 2.0 : 3.0);
    prof_end(st, ev, (mode == OP_JACOBI || mode == OP_JACOBI0) ? PC_JACOBI : (mode == OP_RESID && sizeof(T) == 8) ? PC_RESID64 : PC_RESID,
             nb * sizeof(T) * lv.ncells, lv.ncells);
    return AMR_OK;
  }
  if (D == 3 && !TR && bc == nullptr && (vmask == nullptr || mode == OP_RESID) && zc_eligible(lv, 2)) {
    // z-chunked marching path; rows per thread from the autotuner's table
    const int R = (tile_rows_for(lv, sizeof(T)) == 4 && zc_eligible(lv, 4)) ? 4 : 2;
    const T A = T(alpha), B = T(beta), O = T(omega);
#define LAUNCH_ZC(M)                                                                                    \
  do {                                                                                                  \
    if (R == 4) launch_zc<T, M, 4>(lv, x, f, out, A, B, O, vmask, st);                                  \
    else launch_zc<T, M, 2>(lv, x, f, out, A, B, O, vmask, st);                                         \
  } while (0)
    switch (mode) {
      case OP_APPLY: LAUNCH_ZC(OP_APPLY); break;
      case OP_RESID: LAUNCH_ZC(OP_RESID); break;
      case OP_JACOBI: LAUNCH_ZC(OP_JACOBI); break;
      default: LAUNCH_ZC(OP_JACOBI0);
    }
#undef LAUNCH_ZC
    const double nb = mode == OP_JACOBI0 ? 2.0 : (mode == OP_APPLY ? 2.0 : 3.0);
    prof_end(st, ev, (mode == OP_JACOBI || mode == OP_JACOBI0) ? PC_JACOBI : (mode == OP_RESID && sizeof(T) == 8) ? PC_RESID64 : PC_RESID,
             nb * sizeof(T) * lv.ncells, lv.ncells);
    return launch_check();
  }
  if (D == 3 && !TR && bc == nullptr) {
    // z-marching 3-D path (homogeneous physical data)
    const int tx = (lv.maxn[0] + MZ_TX - 1) / MZ_TX, ty = (lv.maxn[1] + MZ_TY - 1) / MZ_TY;
    const int nz = lv.maxn[2];
    int nzc = std::max(1, std::min((2048 + tx * ty - 1) / (tx * ty), std::max(1, nz / 4)));
    const int kz = (nz + nzc - 1) / nzc;
    nzc = (nz + kz - 1) / kz;
    dim3 grid(tx, ty, nzc * lv.npatch);
    dim3 block(MZ_TX, MZ_TY, 1);
    const T A = T(alpha), B = T(beta), O = T(omega);
    switch (mode) {
      case OP_APPLY: launch(k_level_op3d_march<T, OP_APPLY>, grid, block, 0, st, lv, nzc, kz, x, f, out, A, B, O, vmask); break;
      case OP_RESID: launch(k_level_op3d_march<T, OP_RESID>, grid, block, 0, st, lv, nzc, kz, x, f, out, A, B, O, vmask); break;
      case OP_JACOBI: launch(k_level_op3d_march<T, OP_JACOBI>, grid, block, 0, st, lv, nzc, kz, x, f, out, A, B, O, vmask); break;
      default: launch(k_level_op3d_march<T, OP_JACOBI0>, grid, block, 0, st, lv, nzc, kz, x, f, out, A, B, O, vmask);
    }
    const double nb = mode == OP_JACOBI0 ? 2.0 : (mode == OP_APPLY ? 2.0 : 3.0);
    prof_end(st, ev, (mode == OP_JACOBI || mode == OP_JACOBI0) ? PC_JACOBI : (mode == OP_RESID && sizeof(T) == 8) ? PC_RESID64 : PC_RESID,
             nb * sizeof(T) * lv.ncells, lv.ncells);
    return launch_check();
  }
  switch (mode) {
    case OP_APPLY:
      launch(k_level_op<T, D, OP_APPLY, TR>, g.grid, g.block, 0, st, lv, g.nby, x, f, out, bc, T(alpha), T(beta), T(omega), vmask);
      break;
    case OP_RESID:
      launch(k_level_op<T, D, OP_RESID, TR>, g.grid, g.block, 0, st, lv, g.nby, x, f, out, bc, T(alpha), T(beta), T(omega), vmask);
      break;
    case OP_JACOBI:
      launch(k_level_op<T, D, OP_JACOBI, TR>, g.grid, g.block, 0, st, lv, g.nby, x, f, out, bc, T(alpha), T(beta), T(omega), vmask);
      break;
    default:
      launch(k_level_op<T, D, OP_JACOBI0, TR>, g.grid, g.block, 0, st, lv, g.nby, x, f, out, bc, T(alpha), T(beta), T(omega), vmask);
  }
  // algorithmic bytes: Jacobi reads x, f and writes the sweep (the first sweep reads f
  // only); residual reads x, f and writes r; apply reads x and writes the result
  const double nb = mode == OP_JACOBI0 ? 2.0 : (mode == OP_APPLY ? 2.0 : 3.0);
  prof_end(st, ev, (mode == OP_JACOBI || mode == OP_JACOBI0) ? PC_JACOBI : (mode == OP_RESID && sizeof(T) == 8) ? PC_RESID64 : PC_RESID,
             nb * sizeof(T) * lv.ncells, lv.ncells);
  return launch_check();
}

template <typename T, int D, bool TR = false>
amr_status restrict_blocks(const LevelView& fine, const LevelView& crs, const XferBlock* blocks, int nblocks,
                           const int xmax[3], bool resid, const T* xf, const T* ff, T* outc, double alpha,
                           double beta, cudaStream_t st) {
  if (nblocks == 0) return AMR_OK;
  const int nby = (xmax[1] + BY - 1) / BY;
  dim3 grid((xmax[0] + BX - 1) / BX, nby * (D == 3 ? xmax[2] : 1), nblocks);
  dim3 block(BX, BY, 1);
  cudaEvent_t ev;
  prof_begin(st, &ev);
  if (resid && D == 2)
    launch(k_restrict2d_resid<T, TR>, grid, block, 0, st, fine, crs, blocks, xf, ff, outc, T(alpha), T(beta));
  else if (resid)
    launch(k_restrict<T, D, true, TR>, grid, block, 0, st, fine, crs, blocks, xf, ff, outc, T(alpha), T(beta), nby);
  else
    launch(k_restrict<T, D, false>, grid, block, 0, st, fine, crs, blocks, xf, ff, outc, T(alpha), T(beta), nby);
  const double cc = (double)xmax[0] * xmax[1] * (D == 3 ? xmax[2] : 1) * nblocks;
  prof_end(st, ev, PC_RESTRICT, ((resid ? 2.0 : 1.0) * (1 << D) + 1.0) * sizeof(T) * cc, cc * (1 << D));
  return launch_check();
}

template <typename T, int D>
amr_status prolong_blocks(const LevelView& fine, const LevelView& crs, const XferBlock* blocks, int nblocks,
                          const int xmax[3], const T* xc, T* xf, T* xf2, cudaStream_t st) {
  if (nblocks == 0) return AMR_OK;
  cudaEvent_t ev;
  prof_begin(st, &ev);
  if (D == 2) {
    dim3 grid((xmax[0] + BX - 1) / BX, (xmax[1] + BY - 1) / BY, nblocks);
    launch(k_prolong2d<T>, grid, dim3(BX, BY, 1), 0, st, fine, crs, blocks, xc, xf, xf2);
  } else {
    // 32-bit offsets inside the padded patches (a 3-D patch beyond 2^31 elements takes the
    // generic kernel)
    const long long fel = (long long)(fine.maxn[0] + 2 * NG + 3) * (fine.maxn[1] + 2 * NG) * (fine.maxn[2] + 2 * NG);
    // large grids: four fine cells per thread along z, the face layer in its own launch (a few
    // blocks per face); small grids: one cell per thread with the face cells inline
    const bool large = (long long)xmax[0] * xmax[1] * xmax[2] >= 64LL * 64 * 64;
    const int pz = large ? 4 : 1;
    const int nzc = (2 * xmax[2] + pz - 1) / pz;
    if (fel < (1LL << 31) && (long long)nzc * nblocks <= 65535) {
      dim3 grid((2 * xmax[0] + BX - 1) / BX, (2 * xmax[1] + BY - 1) / BY, nzc * nblocks);
      if (large) {
        // by coarse parent (32 x 8 coarse cells a block, one coarse plane), the face layer by the shell
        dim3 pgrid((xmax[0] + BX - 1) / BX, (xmax[1] + BY - 1) / BY, xmax[2] * nblocks);
        launch(k_prolong3d_par<T>, pgrid, dim3(BX, BY, 1), 0, st, fine, crs, blocks, xmax[2], xc, xf, xf2);
        if (const amr_status s1 = launch_check(); s1 != AMR_OK) return s1;
        const long long face = 4LL * std::max({xmax[0] * xmax[1], xmax[1] * xmax[2], xmax[0] * xmax[2]});
        const unsigned gx = (unsigned)std::min<long long>((face + 255) / 256, 64);
        launch(k_prolong3d_shell<T>, dim3(gx, 6, nblocks), 256, 0, st, fine, crs, blocks, xc, xf, xf2);
      } else {
        launch(k_prolong3d<T, true, 1>, grid, dim3(BX, BY, 1), 0, st, fine, crs, blocks, nzc, xc, xf, xf2);
      }
    } else {
      const int fy = 2 * xmax[1];
      const int nby = (fy + BY - 1) / BY;
      dim3 grid((2 * xmax[0] + BX - 1) / BX, nby * (D == 3 ? 2 * xmax[2] : 1), nblocks);
      launch(k_prolong<T, D>, grid, dim3(BX, BY, 1), 0, st, fine, crs, blocks, xc, xf, xf2, nby);
    }
  }
  const double cc = (double)xmax[0] * xmax[1] * (D == 3 ? xmax[2] : 1) * nblocks;
  prof_end(st, ev, PC_PROLONG, (1.0 + (1 << D) * (xf2 ? 4.0 : 2.0)) * sizeof(T) * cc, cc * (1 << D));
  return launch_check();
}

template <typename T, int D>
amr_status cfi_fill(const amr_hierarchy* h, int l, const T* xc, T* xf, bool zero, cudaStream_t st) {
  const DeviceLists& dl = h->lev[l].dev;
  if (dl.ncfi == 0) return AMR_OK;
  const int nt = 128;
  if (dl.ncfig > 0) {  // ratio 2: by coarse parent
    launch(k_cfi_grp<T, D>, (unsigned)((dl.ncfig + nt - 1) / nt), nt, 0, st, dl.cfig, dl.ncfig, dl.cfi_side,
           h->lev[l - 1].d_patches, xc, xf, zero ? 1 : 0);
    return launch_check();
  }
  launch(k_cfi<T, D>, (unsigned)((dl.ncfi + nt - 1) / nt), nt, 0, st, dl.cfi, dl.ncfi, dl.cfi_side, h->lev[l - 1].d_patches,
                                                                  h->r, xc, xf, zero ? 1 : 0);
  return launch_check();
}

template <typename T>
amr_status copy_fill(const amr_hierarchy* h, int l, T* x, cudaStream_t st) {
  const DeviceLists& dl = h->lev[l].dev;
  if (dl.ncopy == 0) return AMR_OK;
  const int nt = 128;
  launch(k_copy<T>, (unsigned)((dl.ncopy + nt - 1) / nt), nt, 0, st, dl.copy, dl.ncopy, x);
  return launch_check();
}

template <typename T>
struct P3 {
  const T* p[3];
};

template <typename T, int D>
__global__ void k_reflux_p3(LevelView crs, LevelView fine, const RefluxEntry* __restrict__ list, long long n,
                            P3<T> xcs, P3<T> xfs, P3<T> bcs, T* __restrict__ out, T coef, int kind);

template <typename T, int D>
amr_status reflux(const amr_hierarchy* h, int l, const LevelView& crs, const LevelView& fine, P3<T> xc, P3<T> xf,
                  P3<T> bcs, T* out, double coef, int kind, cudaStream_t st) {
  const DeviceLists& dl = h->lev[l].dev;
  if (dl.nreflux == 0) return AMR_OK;
  const int nt = 128;
  launch(k_reflux_p3<T, D>, (unsigned)((dl.nreflux + nt - 1) / nt), nt, 0, st, crs, fine, dl.reflux, dl.nreflux, xc, xf,
                                                                         bcs, out, T(coef), kind);
  return launch_check();
}

template <typename S, typename T, int D>
amr_status axpy(const LevelView& lv, const S* x, T* y, T* y2, double a, cudaStream_t st) {
  Geo g = geo_of(lv);
  launch(k_axpy<S, T, D>, g.grid, g.block, 0, st, lv, g.nby, x, y, y2, T(a));
  return launch_check();
}

template <typename S, typename T, int D>
amr_status convert(const LevelView& lv, const S* x, T* y, cudaStream_t st) {
  Geo g = geo_of(lv);
  launch(k_convert<S, T, D>, g.grid, g.block, 0, st, lv, g.nby, x, y);
  return launch_check();
}


}  // namespace

// reflux kernel with by-value pointer triples (defined outside the anonymous namespace
// declaration above so that it can be instantiated)
namespace {
// Refluxing (COH-3) of one coarse cell: its flux through every coarse-fine face replaced by
// the mean of the fine fluxes.  KIND 0: the derivative flux of L (1/12, -15/12, 15/12, -1/12
// divided by h); KIND 1: the face value of D (-1/12, 7/12, 7/12, -1/12).  Reciprocals of h
// instead of divisions: FP64 division is slow on this part.
template <typename T, int D, int KIND>
__device__ __forceinline__ void reflux_cell(const LevelView& crs, const LevelView& fine, const RefluxEntry& e,
                                            const P3<T>& xcs, const P3<T>& xfs, const P3<T>& bcs, T* __restrict__ out,
                                            T coef) {
  constexpr double FC[2][4] = {{1.0 / 12.0, -15.0 / 12.0, 15.0 / 12.0, -1.0 / 12.0},
                               {-1.0 / 12.0, 7.0 / 12.0, 7.0 / 12.0, -1.0 / 12.0}};
  const PatchDesc cp = crs.patches[e.cpatch];
  const T ihc = KIND == 0 ? pick<T>(crs.invh, crs.invh_f) : T(1);
  const T ihf = KIND == 0 ? pick<T>(fine.invh, fine.invh_f) : T(1);
  T corr = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (!(e.faces & (1 << (2 * d + side)))) continue;
      const int comp = KIND == 0 ? 0 : d;
      const T* xc = xcs.p[comp];
      const T* xf = xfs.p[comp];
      int own[3] = {e.g[0] - cp.lo[0], e.g[1] - cp.lo[1], e.g[2] - cp.lo[2]};
      if (side == 0) own[d] -= 1;
      T Fc = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int cc[3] = {own[0], own[1], own[2]};
        cc[d] += q - 1;
        Fc += T(FC[KIND][q]) * read_nb<T, D>(xc, cp, crs, bcs.p[comp], cc[0], cc[1], cc[2], d);
      }
      const PatchDesc fp = fine.patches[e.fpatch[2 * d + side]];
      T Fs = T(0);
      const int t1d = (d == 0) ? 1 : 0;
      const int t2d = (d == 2) ? 1 : 2;
#pragma unroll
      for (int t2 = 0; t2 < (D == 3 ? 2 : 1); ++t2)
#pragma unroll
        for (int t1 = 0; t1 < 2; ++t1) {
          int gf[3] = {0, 0, 0};
          gf[d] = side == 1 ? 2 * (e.g[d] + 1) - 1 : 2 * e.g[d] - 1;
          gf[t1d] = 2 * e.g[t1d] + t1;
          if (D == 3) gf[t2d] = 2 * e.g[t2d] + t2;
          const int cf[3] = {gf[0] - fp.lo[0], gf[1] - fp.lo[1], gf[2] - fp.lo[2]};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int cc[3] = {cf[0], cf[1], cf[2]};
            cc[d] += q - 1;
            Fs += T(FC[KIND][q]) * xf[poff(fp, cc[0], cc[1], cc[2])];
          }
        }
      const T Fbar = Fs * T(D == 3 ? 0.25 : 0.5);
      corr += T(side == 1 ? 1 : -1) * (Fbar * ihf - Fc * ihc);
    }
  out[e.coff] += coef * corr * pick<T>(crs.invh, crs.invh_f);
}

template <typename T, int D>
__global__ void k_reflux_p3(LevelView crs, LevelView fine, const RefluxEntry* __restrict__ list, long long n,
                            P3<T> xcs, P3<T> xfs, P3<T> bcs, T* __restrict__ out, T coef, int kind) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const RefluxEntry e = list[t];
  if (kind == 0) reflux_cell<T, D, 0>(crs, fine, e, xcs, xfs, bcs, out, coef);
  else reflux_cell<T, D, 1>(crs, fine, e, xcs, xfs, bcs, out, coef);
}

// ---------------------------------------------------------------- scratch management
template <typename T>
Scratch<T>& scratch(amr_operator* op);
template <>
Scratch<double>& scratch<double>(amr_operator* op) { return op->s64; }
template <>
Scratch<float>& scratch<float>(amr_operator* op) { return op->s32; }

template <typename T, int D>
amr_status autotune_tiles(amr_operator* op, cudaStream_t st);
template <typename T>
amr_status blk_attrs();

template <typename T>
amr_status ensure_scratch(amr_operator* op) {
  Scratch<T>& S = scratch<T>(op);
  if (S.ready) return AMR_OK;
  const amr_hierarchy* h = op->h;
  const size_t n = (size_t)h->nelems;
  TRY(dalloc(&S.E, n));
  TRY(dalloc(&S.R, n));
  TRY(dalloc(&S.T1, n));
  TRY(dalloc(&S.T2, n));
  TRY(dalloc(&S.X, n));
  TRY(dalloc(&S.rin, n));
  TRY(dalloc(&S.Z, n));
  TRY(dalloc(&S.W, n));
  TRY(dalloc(&S.Y, n));
  CK(cudaMemset(S.Y, 0, n * sizeof(T)));
  CK(cudaMemset(S.Z, 0, n * sizeof(T)));
  CK(cudaMemset(S.W, 0, n * sizeof(T)));
  CK(cudaMemset(S.E, 0, n * sizeof(T)));
  CK(cudaMemset(S.R, 0, n * sizeof(T)));
  CK(cudaMemset(S.T1, 0, n * sizeof(T)));
  CK(cudaMemset(S.T2, 0, n * sizeof(T)));
  CK(cudaMemset(S.X, 0, n * sizeof(T)));
  CK(cudaMemset(S.rin, 0, n * sizeof(T)));
  S.mx.assign(h->mg.size(), nullptr);
  S.mb.assign(h->mg.size(), nullptr);
  S.mt.assign(h->mg.size(), nullptr);
  for (size_t m = 1; m < h->mg.size(); ++m) {
    const size_t q = (size_t)h->mg[m].nelems;
    TRY(dalloc(&S.mx[m], q));
    TRY(dalloc(&S.mb[m], q));
    TRY(dalloc(&S.mt[m], q));
    CK(cudaMemset(S.mx[m], 0, q * sizeof(T)));
    CK(cudaMemset(S.mb[m], 0, q * sizeof(T)));
    CK(cudaMemset(S.mt[m], 0, q * sizeof(T)));
  }
  S.ready = true;
  // choose the tiled kernels' rows per thread for every grid this operator smooths
  if (op->h->D == 2) {
    if constexpr (sizeof(T) == 4) TRY(blk_attrs<T>());
    TRY((autotune_tiles<T, 2>(op, 0)));
  } else {
    TRY((autotune_tiles<T, 3>(op, 0)));
  }
  return AMR_OK;
}

template <typename T>
void free_scratch(Scratch<T>& S) {
  cudaFree(S.E); cudaFree(S.R); cudaFree(S.T1); cudaFree(S.T2); cudaFree(S.X); cudaFree(S.rin);
  cudaFree(S.Z); cudaFree(S.W); cudaFree(S.Y);
  for (auto p : S.mx) cudaFree(p);
  for (auto p : S.mb) cudaFree(p);
  for (auto p : S.mt) cudaFree(p);
  S = Scratch<T>();
}

template <typename T, int D>
amr_status autotune_tiles(amr_operator* op, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  // (grid, x, f, out): three distinct buffers, so that the timed sweeps move the bytes a real
  // sweep moves (a grid whose fields exceed L2 must not be timed from L2)
  struct Case {
    LevelView lv;
    T *x, *f, *o;
  };
  std::vector<Case> cases;
  for (int l = 0; l < h->L; ++l) cases.push_back({level_view(h, l, op->bc), S.T1, S.R, S.T2});
  for (size_t m = 1; m < h->mg.size(); ++m) cases.push_back({mg_view(h, (int)m, op->bc), S.mx[m], S.mb[m], S.mt[m]});
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (auto& c : cases) {
    const LevelView& lv = c.lv;
    std::vector<int> variants = D == 3 ? std::vector<int>{2} : std::vector<int>{1, 2, 4};
    if (D == 3 && zc_eligible(lv, 4)) variants.push_back(4);
    if (D == 3 && sw_eligible(lv)) variants.push_back(TILE_BULK);
    if (variants.size() < 2) continue;  // nothing to choose
    const long long key = tile_key(lv, sizeof(T));
    {
      std::lock_guard<std::mutex> lock(g_tile_mu);
      bool known = false;
      for (const auto& e : g_tile_table) known = known || e.first == key;
      if (known) continue;
    }
    float best = 1e30f;
    int best_rows = D == 3 ? 2 : 1;
    for (int rows : variants) {
      {
        std::lock_guard<std::mutex> lock(g_tile_mu);
        g_tile_table.push_back({key, rows});
      }
      for (int rep = 0; rep < 2; ++rep) {  // warm-up, then timed
        CK(cudaEventRecord(a, st));
        for (int it = 0; it < 4; ++it)
          TRY((level_op<T, D>(OP_JACOBI, lv, c.x, c.f, c.o, nullptr, op->alpha, op->beta, 2.0 / 3.0, nullptr, st)));
        CK(cudaEventRecord(b, st));
      }
      CK(cudaEventSynchronize(b));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, a, b));
      {
        std::lock_guard<std::mutex> lock(g_tile_mu);
        g_tile_table.pop_back();
      }
      // a larger tile (or the bulk-copy kernel) must win by 5 %: timing back-to-back sweeps
      // flatters it (warmer L2)
      if (ms < 0.95f * best) { best = ms; best_rows = rows; }
    }
    std::lock_guard<std::mutex> lock(g_tile_mu);
    g_tile_table.push_back({key, best_rows});
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return AMR_OK;
}

// ---------------------------------------------------------------- smoothing
// nsweeps weighted-Jacobi sweeps on one level from x = 0 (first sweep closed form), the
// result ends in ``a`` (b is the other ping-pong buffer).  Copy ghosts are refreshed
// before every sweep; CF ghosts of a and b must already be zero.
template <typename T, int D, bool TR = false>
amr_status smooth_from_zero(const amr_hierarchy* h, int l, const LevelView& lv, const T* f, T* a, T* b, int nsweeps,
                            double alpha, double beta, double omega, bool amr_level, cudaStream_t st) {
  if (nsweeps <= 0) return AMR_OK;
  T* cur = (nsweeps % 2 == 1) ? a : b;
  T* oth = (cur == a) ? b : a;
  TRY(level_op<T, D, TR>(OP_JACOBI0, lv, nullptr, f, cur, nullptr, alpha, beta, omega, nullptr, st));
  for (int s = 1; s < nsweeps; ++s) {
    if (amr_level) TRY(copy_fill<T>(h, l, cur, st));
    TRY(level_op<T, D, TR>(OP_JACOBI, lv, cur, f, oth, nullptr, alpha, beta, omega, nullptr, st));
    std::swap(cur, oth);
  }
  return AMR_OK;
}

// nsweeps sweeps starting from the values in a; result in a (copy back if odd).
template <typename T, int D, bool TR = false>
amr_status smooth_from(const amr_hierarchy* h, int l, const LevelView& lv, const T* f, T* a, T* b, int nsweeps,
                       double alpha, double beta, double omega, bool amr_level, cudaStream_t st) {
  T* cur = a;
  T* oth = b;
  for (int s = 0; s < nsweeps; ++s) {
    if (amr_level) TRY(copy_fill<T>(h, l, cur, st));
    TRY(level_op<T, D, TR>(OP_JACOBI, lv, cur, f, oth, nullptr, alpha, beta, omega, nullptr, st));
    std::swap(cur, oth);
  }
  if (cur != a) {
    // odd count: bring the result back into a (interior cells)
    TRY(convert<T, T, D>(lv, cur, a, st));
  }
  return AMR_OK;
}

// ---------------------------------------------------------------- fused coarse V-cycle
constexpr size_t CMG_SMEM_BUDGET = 200 * 1024;

inline PatchDesc smem_patch(const MgGrid& g, int D) {
  PatchDesc p{};
  p.off = 0;
  p.sy = g.n[0] + 2 * NG;
  p.sz = (D == 3) ? p.sy * (g.n[1] + 2 * NG) : 0;
  for (int e = 0; e < 3; ++e) { p.n[e] = g.n[e]; p.lo[e] = 0; }
  return p;
}
inline long long smem_elems(const MgGrid& g, int D) {
  const PatchDesc p = smem_patch(g, D);
  return (D == 3) ? p.sz * (g.n[2] + 2 * NG) : p.sy * (g.n[1] + 2 * NG);
}

// First grid of the fused part: the finest m such that grids m..coarsest fit together in the
// shared-memory budget (three arrays each) and number at most CMG_MAX.
template <typename T, int D, bool TR = false>
amr_status fused_config(amr_operator* op, int& m0, size_t& bytes) {
  const int pi = sizeof(T) == 4 ? 0 : 1;
  const int ti = TR ? 1 : 0;
  if (op->cmg_m0[ti][pi] >= 0) { m0 = op->cmg_m0[ti][pi]; bytes = op->cmg_bytes[ti][pi]; return AMR_OK; }
  const amr_hierarchy* h = op->h;
  const int M = (int)h->mg.size() - 1;
  size_t acc = 0;
  m0 = M + 1;
  for (int m = M; m >= 0 && M - m + 1 <= CMG_MAX; --m) {
    const size_t need = acc + 3 * (size_t)smem_elems(h->mg[m], D) * sizeof(T);
    if (need > CMG_SMEM_BUDGET) break;
    acc = need;
    m0 = m;
  }
  bytes = acc;
  if (m0 <= M) {
    CK(cudaFuncSetAttribute(k_coarse_mg<T, D, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }
  op->cmg_m0[ti][pi] = m0;
  op->cmg_bytes[ti][pi] = bytes;
  return AMR_OK;
}

static_assert(sizeof(CoarseMG) < 30000, "kernel parameter block too large");

template <typename T, int D, bool TR = false>
amr_status fused_coarse(amr_operator* op, const amr_solver_params& p, int m0, size_t bytes, const T* b, T* x,
                        cudaStream_t st) {
  amr_hierarchy* h = op->h;
  const int M = (int)h->mg.size() - 1;
  CoarseMG cm{};
  cm.ng = M - m0 + 1;
  cm.nu1 = p.nu1;
  cm.nu2 = p.nu2;
  cm.nbot = op->nbot;
  cm.ldb = op->ldb;
  cm.minv = TR ? op->d_binvT : op->d_binv;
  cm.gp = h->mg[m0].patch;
  long long off = 0;
  for (int q = 0; q < cm.ng; ++q) {
    const MgGrid& g = h->mg[m0 + q];
    cm.lv[q] = mg_view(h, m0 + q, op->bc);
    cm.sp[q] = smem_patch(g, D);
    const long long e = smem_elems(g, D);
    cm.offx[q] = (int)off; off += e;
    cm.offb[q] = (int)off; off += e;
    cm.offt[q] = (int)off; off += e;
  }
  launch(k_coarse_mg<T, D, TR>, 1, 1024, bytes, st, cm, b, x, T(op->alpha), T(op->beta), T(p.omega));
  return launch_check();
}

// ---------------------------------------------------------------- temporally blocked legs
constexpr int BLK_MAX_NU = 6;

// tile edge: small grids need many blocks, large grids a small halo share
inline int blk_tile(const int* n) { return (long long)n[0] * n[1] >= 1024LL * 1024 ? 32 : 16; }

// dynamic shared memory of a blocked leg: three region arrays with two ghost layers
template <typename T>
size_t blk_smem(const int* n, int halo) {
  const int t = blk_tile(n);
  const long long w = std::min(t + 2 * halo, n[0]) + 2 * NG;
  const long long hh = std::min(t + 2 * halo, n[1]) + 2 * NG;
  return (size_t)(3 * w * hh) * sizeof(T);
}

// Blocked legs with compile-time region bounds (nu <= 4, tiles of 16 or 32): the down leg's
// region is the tile plus 2 nu + 2 cells per side, the up leg's and the post-smoothing's the
// tile plus 2 nu; other shapes take the runtime-bounded kernels.
constexpr int BLK_FX_NU = 4;
template <typename T, typename... A>
void launch_down2d(int tt, int nu, dim3 grid, size_t smem, cudaStream_t st, A&&... a) {
  if (nu <= BLK_FX_NU && tt == 16) launch(k_mg_down2d<T, 16 + 4 * BLK_FX_NU + 4, 16, 512>, grid, dim3(32, 16, 1), smem, st, a...);
  else if (nu <= BLK_FX_NU && tt == 32) launch(k_mg_down2d<T, 32 + 4 * BLK_FX_NU + 4, 32>, grid, dim3(32, 8, 1), smem, st, a...);
  else launch(k_mg_down2d<T>, grid, dim3(32, 8, 1), smem, st, a...);
}
template <typename T, typename... A>
void launch_up2d(int tt, int nu, dim3 grid, size_t smem, cudaStream_t st, A&&... a) {
  if (nu <= BLK_FX_NU && tt == 16) launch(k_mg_up2d<T, 16 + 4 * BLK_FX_NU, 16, 512>, grid, dim3(32, 16, 1), smem, st, a...);
  else if (nu <= BLK_FX_NU && tt == 32) launch(k_mg_up2d<T, 32 + 4 * BLK_FX_NU, 32>, grid, dim3(32, 8, 1), smem, st, a...);
  else launch(k_mg_up2d<T>, grid, dim3(32, 8, 1), smem, st, a...);
}
template <typename T, typename... A>
void launch_post2d(int tt, int nu, dim3 grid, size_t smem, cudaStream_t st, A&&... a) {
  if (nu <= BLK_FX_NU && tt == 16) launch(k_amr_post2d<T, 16 + 4 * BLK_FX_NU, 16, 512>, grid, dim3(32, 16, 1), smem, st, a...);
  else if (nu <= BLK_FX_NU && tt == 32) launch(k_amr_post2d<T, 32 + 4 * BLK_FX_NU, 32>, grid, dim3(32, 8, 1), smem, st, a...);
  else launch(k_amr_post2d<T>, grid, dim3(32, 8, 1), smem, st, a...);
}
// shared memory of a blocked launch: the compile-time region bound when that kernel runs
template <typename T>
size_t blk_smem_fx(const int* n, int nu, bool down) {
  const int tt = blk_tile(n);
  if (nu > BLK_FX_NU) return blk_smem<T>(n, down ? 2 * nu + 2 : 2 * nu);
  const int rm = tt + (down ? 4 * BLK_FX_NU + 4 : 4 * BLK_FX_NU) + 2 * NG;
  return (size_t)3 * rm * rm * sizeof(T);
}

template <typename T>
amr_status blk_attrs() {
  static bool done = false;
  if (done) return AMR_OK;
  const int bytes = 200 * 1024;
  CK(cudaFuncSetAttribute(k_mg_down2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_mg_up2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_amr_post2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_mg_coarse2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_mg_coarse2d_sq<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_mg_coarse2d_sq<T, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done = true;
  return AMR_OK;
}

// first grid of the one-block coarse V-cycle: every grid from it down fits a block (at most
// 64 cells per dimension, CB_MAX grids, shared-memory budget); -1 when none below the top
inline int coarse_block_m0(const amr_hierarchy* h, size_t& bytes) {
  const int M = (int)h->mg.size() - 1;
  int m0 = -1;
  size_t acc = 0;
  for (int m = M; m >= 0 && M - m + 1 <= CB_MAX; --m) {
    const MgGrid& g = h->mg[m];
    if (g.n[0] > BLK_MAX_REGION || g.n[1] > BLK_MAX_REGION) break;
    const size_t need = acc + 3 * (size_t)(g.n[0] + 2 * NG) * (g.n[1] + 2 * NG) * sizeof(float);
    if (need > 200 * 1024) break;
    acc = need;
    m0 = m;
  }
  bytes = acc;
  return m0 < M ? m0 : -1;
}

// descriptor of the one-block coarse V-cycle from grid m0 down
inline CoarseBlock2D make_coarse_block(const amr_operator* op, const amr_solver_params& p, int m0) {
  const amr_hierarchy* h = op->h;
  const int M = (int)h->mg.size() - 1;
  CoarseBlock2D cb{};
  cb.ng = M - m0 + 1;
  cb.nu1 = p.nu1;
  cb.nu2 = p.nu2;
  cb.nbot = op->nbot;
  cb.ldb = op->ldb;
  cb.minv = op->d_binv;
  cb.gp = h->mg[m0].patch;
  int off = 0;
  for (int q = 0; q < cb.ng; ++q) {
    const MgGrid& g = h->mg[m0 + q];
    const int e = (g.n[0] + 2 * NG) * (g.n[1] + 2 * NG);
    cb.offx[q] = off; off += e;
    cb.offt[q] = off; off += e;
    cb.offb[q] = off; off += e;
    cb.lv[q] = mg_view(h, m0 + q, op->bc);
    cb.ood[q] = p.omega / (op->alpha - 60.0 * op->beta * cb.lv[q].inv12h2);
  }
  return cb;
}

// 64 or 48 when the pyramid from m0 is square N0, N0/2, ... down to the compile-time-size
// kernel's bottom grid, else 0
inline int square_pyramid(const amr_operator* op, int m0, int ng) {
  const amr_hierarchy* h = op->h;
  for (int n0 : {64, 48}) {
    bool ok = true;
    for (int q = 0; q < ng && ok; ++q) {
      const MgGrid& g = h->mg[m0 + q];
      ok = g.n[0] == (n0 >> q) && g.n[1] == (n0 >> q);
    }
    const int nb = n0 == 64 ? sq_bottom<64, 64>() : sq_bottom<48, 48>();
    const int ngr = 1 + (n0 == 64 ? sq_depth<64, sq_bottom<64, 64>()>() : sq_depth<48, sq_bottom<48, 48>()>());
    if (ok && ng == ngr && op->nbot == nb * nb) return n0;
  }
  return 0;
}

template <typename T, int D>
amr_status coarse_block(amr_operator* op, const amr_solver_params& p, int m0, size_t bytes, const T* b, T* x,
                        cudaStream_t st) {
  const CoarseBlock2D cb = make_coarse_block(op, p, m0);
  // square pyramids N0, N0/2, ... with N0 = 64 or 48 take the compile-time-size kernel
  const int sq = square_pyramid(op, m0, cb.ng);
  cudaEvent_t ev;
  prof_begin(st, &ev);
  if (sq == 64)
    launch(k_mg_coarse2d_sq<T, 64>, 1, dim3(32, 32, 1), sizeof(T) * sq_total<64, 64>(), st, cb, b, x, T(op->alpha),
           T(op->beta), T(p.omega));
  else if (sq == 48)
    launch(k_mg_coarse2d_sq<T, 48>, 1, dim3(32, 32, 1), sizeof(T) * sq_total<48, 48>(), st, cb, b, x, T(op->alpha),
           T(op->beta), T(p.omega));
  else
    launch(k_mg_coarse2d<T>, 1, dim3(32, 32, 1), bytes, st, cb, b, x, T(op->alpha), T(op->beta), T(p.omega));
  TRY(launch_check());
  prof_end(st, ev, PC_COARSE, 2.0 * sizeof(T) * (double)op->h->mg[m0].n[0] * op->h->mg[m0].n[1]);  // read f, write x
  return AMR_OK;
}

// ---------------------------------------------------------------- cube coarse V-cycle (3-D)
// Grid m of the level-0 pyramid starts the compile-time-size cube kernel: it and the grids
// below are 16^3, 8^3 and the 4^3 bottom (one block per replica of a stacked batch).
constexpr int CUBE_N0 = 16;
inline bool cube_pyramid(const amr_operator* op, int m) {
  const amr_hierarchy* h = op->h;
  constexpr int ng = cu_ngrids<CUBE_N0>();
  if (h->D != 3 || m + ng != (int)h->mg.size()) return false;
  for (int q = 0; q < ng; ++q) {
    const MgGrid& g = h->mg[m + q];
    for (int e = 0; e < 3; ++e)
      if (g.n[e] != (CUBE_N0 >> q)) return false;
  }
  constexpr int nb = cu_bottom<CUBE_N0, CUBE_N0>();
  return op->nbot == nb * nb * nb;
}

template <typename T>
amr_status cube_coarse(amr_operator* op, const amr_solver_params& p, int m0, const T* b, T* x, cudaStream_t st) {
  static std::mutex mu;
  static bool done[64] = {false};
  constexpr size_t smem = sizeof(T) * cu_total<CUBE_N0, CUBE_N0>();
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && !done[dev]) {
      CK(cudaFuncSetAttribute(k_mg_coarse3d_cube<T, CUBE_N0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      done[dev] = true;
    }
  }
  const amr_hierarchy* h = op->h;
  CubeBlock cb{};
  cb.nu1 = p.nu1;
  cb.nu2 = p.nu2;
  cb.nbot = op->nbot;
  cb.ldb = op->ldb;
  cb.minv = op->d_binv;
  cb.gp = h->mg[m0].patch;
  const LevelView l0 = mg_view(h, m0, op->bc);
  for (int f = 0; f < 6; ++f) cb.bcm |= (l0.bc[f] & 1) << f;
  cb.cstride = h->ncomp > 1 ? h->mg[m0].cstride : 0;
  cb.active = l0.active;
  const float alpha = (float)op->alpha, beta = (float)op->beta, omega = (float)p.omega;
  cb.alpha = alpha;
  for (int q = 0; q < cu_ngrids<CUBE_N0>(); ++q) {
    const LevelView lv = mg_view(h, m0 + q, op->bc);
    const float inv = lv.inv12h2_f;
    cb.binv[q] = beta * inv;
    for (int c = 0; c < 125; ++c) {
      const int cls[3] = {c % 5, (c / 5) % 5, c / 25};
      float acc = -90.0f;
      for (int d = 0; d < 3; ++d)
        if (cls[d]) acc += lv.dcorr_f[2 * d + (cls[d] - 1) / 2][(cls[d] - 1) % 2];
      cb.wt[q][c] = omega / (alpha + beta * inv * acc);
    }
  }
  cudaEvent_t ev;
  prof_begin(st, &ev);
  launch(k_mg_coarse3d_cube<T, CUBE_N0>, h->ncomp, dim3(32, 32, 1), smem, st, cb, b, x);
  TRY(launch_check());
  const double cells = (double)CUBE_N0 * CUBE_N0 * CUBE_N0 * h->ncomp;
  prof_end(st, ev, PC_COARSE, 2.0 * sizeof(T) * cells, cells);  // read f, write x
  return AMR_OK;
}

// ---------------------------------------------------------------- cluster coarse V-cycle (3-D)
// First level-0 multigrid grid from which every grid down to the bottom has at most
// CC_CELLS cells (and there are at most CC_MAX of them, at least one above the bottom); -1
// when there is none.
inline int coarse_cluster_m0(const amr_hierarchy* h) {
  const int M = (int)h->mg.size() - 1;
  int m0 = -1;
  for (int m = M; m >= 0 && M - m + 1 <= CC_MAX; --m) {
    const MgGrid& g = h->mg[m];
    if ((long long)g.n[0] * g.n[1] * g.n[2] > CC_CELLS) break;
    m0 = m;
  }
  return m0 < M ? m0 : -1;
}

// CTAs per cluster: 16 where the device schedules a cluster that large, else 8 (queried
// once per device and kernel)
template <typename T, int D, bool TR>
int coarse_cluster_size() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int cs = 8;
  if (cudaFuncSetAttribute(k_coarse_cluster<T, D, TR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
      cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(CC_THREADS, 1, 1);
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = 16;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = 1;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_cluster<T, D, TR>, &cfg) == cudaSuccess && nclusters >= 1)
      cs = 16;
  }
  cudaGetLastError();
  cache[dev] = cs;
  return cs;
}

template <typename T, int D, bool TR = false>
amr_status coarse_cluster(amr_operator* op, const amr_solver_params& p, int m0, const T* b, T* x, T* t,
                          cudaStream_t st) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  const int M = (int)h->mg.size() - 1;
  CoarseCluster cm{};
  CoarsePtrs<T> ptr{};
  cm.ng = M - m0 + 1;
  cm.nu1 = p.nu1;
  cm.nu2 = p.nu2;
  cm.nbot = op->nbot;
  cm.ldb = op->ldb;
  cm.minv = TR ? op->d_binvT : op->d_binv;
  for (int q = 0; q < cm.ng; ++q) {
    const int m = m0 + q;
    cm.lv[q] = mg_view(h, m, op->bc);
    cm.gp[q] = h->mg[m].patch;
    ptr.x[q] = q == 0 ? x : S.mx[m];
    ptr.b[q] = q == 0 ? const_cast<T*>(b) : S.mb[m];
    ptr.t[q] = q == 0 ? t : S.mt[m];
  }
  const int cs = coarse_cluster_size<T, D, TR>();
  cudaEvent_t ev;
  prof_begin(st, &ev);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(CC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, D, TR>, cm, ptr, T(op->alpha), T(op->beta),
                                           T(p.omega));
  if (e != cudaSuccess && g_launch_err == cudaSuccess) g_launch_err = e;
  TRY(launch_check());
  const MgGrid& g = h->mg[m0];
  const double cells = (double)g.n[0] * g.n[1] * g.n[2];
  prof_end(st, ev, PC_COARSE, 2.0 * sizeof(T) * cells, cells);  // read f, write x of the top grid
  return AMR_OK;
}
static_assert(sizeof(CoarseCluster) + sizeof(CoarsePtrs<double>) < 30000, "kernel parameter block too large");

// ---------------------------------------------------------------- level-0 multigrid
template <typename T, int D, bool TR = false>
amr_status mg_level0(amr_operator* op, const amr_solver_params& p, int m, const T* b, T* x, T* t, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  const int M = (int)h->mg.size() - 1;
  const LevelView lv = mg_view(h, m, op->bc);
  if (p.fuse_coarse == 1 && h->ncomp == 1) {
    int m0;
    size_t bytes;
    TRY((fused_config<T, D, TR>(op, m0, bytes)));
    if (m == m0) return fused_coarse<T, D, TR>(op, p, m0, bytes, b, x, st);
  }
  if constexpr (D == 3) {
    // fuse_coarse = 2: the coarse end of the pyramid in one cluster launch
    if (p.fuse_coarse == 2 && h->ncomp == 1 && m == coarse_cluster_m0(h))
      return coarse_cluster<T, D, TR>(op, p, m, b, x, t, st);
    // default: a 16^3, 8^3, 4^3 coarse end of an FP32 forward V-cycle in one block
    if constexpr (sizeof(T) == 4 && !TR)
      if (p.fuse_coarse == 0 && p.nu1 >= 1 && cube_pyramid(op, m)) return cube_coarse<T>(op, p, m, b, x, st);
  }
  if (m == M) {
    const int n = op->nbot;
    launch(k_bottom<T, D>, h->ncomp, 256, n * sizeof(double), st, TR ? op->d_binvT : op->d_binv, n, op->ldb,
           h->mg[m].patch, b, x, h->mg[m].cstride);
    return launch_check();
  }
  const LevelView cv = mg_view(h, m + 1, op->bc);
  if constexpr (D == 2 && sizeof(T) == 4 && !TR) if (p.temporal_blocking && p.nu1 >= 1 && p.nu1 <= BLK_MAX_NU && p.nu2 <= BLK_MAX_NU) {
    size_t cbytes = 0;
    if (m == coarse_block_m0(h, cbytes)) return coarse_block<T, D>(op, p, m, cbytes, b, x, st);
    // temporally blocked legs (FP32 forward V-cycles: FP64 arithmetic is scarce on this
    // part and the halo recomputation would cost more than the launches it saves): one
    // launch for {nu1 sweeps, residual, restriction} into t, one for {prolongation, nu2
    // sweeps} from t into x
    const MgGrid& g = h->mg[m];
    const MgGrid& gc = h->mg[m + 1];
    const int tt = blk_tile(g.n);
    dim3 grid((g.n[0] + tt - 1) / tt, (g.n[1] + tt - 1) / tt, 1);
    const dim3 blk(32, 8, 1);
    const int hd = 2 * p.nu1 + 2, hu = 2 * p.nu2;
    const double dint = op->alpha - 60.0 * op->beta * lv.inv12h2;  // interior diagonal
    const T ood = T(p.omega / dint);
    const double cells = (double)g.n[0] * g.n[1];
    cudaEvent_t ev;
    prof_begin(st, &ev);
    (void)blk;
    launch_down2d<T>(tt, p.nu1, grid, blk_smem_fx<T>(g.n, p.nu1, true), st, lv, g.patch, gc.patch, tt, tt, hd, p.nu1, b, t,
                     (T*)nullptr, S.mb[m + 1], T(op->alpha), T(op->beta), T(p.omega), ood);
    TRY(launch_check());
    prof_end(st, ev, PC_DOWN, (2.0 + 0.25) * sizeof(T) * cells);  // read f, write x, write coarse f
    TRY(mg_level0<T, D, TR>(op, p, m + 1, S.mb[m + 1], S.mx[m + 1], S.mt[m + 1], st));
    prof_begin(st, &ev);
    launch_up2d<T>(tt, p.nu2, grid, blk_smem_fx<T>(g.n, p.nu2, false), st, lv, cv, g.patch, gc.patch, tt, tt, hu, p.nu2,
                   (const T*)S.mx[m + 1], (const T*)b, (const T*)t, x, T(op->alpha), T(op->beta), T(p.omega), ood);
    TRY(launch_check());
    prof_end(st, ev, PC_UP, (3.0 + 0.25) * sizeof(T) * cells);  // read x, f, coarse x; write x
    return AMR_OK;
  }
  TRY(smooth_from_zero<T, D, TR>(h, 0, lv, b, x, t, p.nu1, op->alpha, op->beta, p.omega, false, st));
  const int xm[3] = {h->mg[m + 1].n[0], h->mg[m + 1].n[1], h->mg[m + 1].n[2]};
  if (D == 3 && !TR && sw_eligible(lv) && lv.maxn[2] % 2 == 0 && tile_rows_for(lv, sizeof(T)) == TILE_BULK) {
    // the residual restriction by the bulk-copy kernel (same arithmetic as k_restrict)
    cudaEvent_t ev;
    prof_begin(st, &ev);
    TRY(launch_sw<T, OP_RESTRICT>(lv, x, b, (T*)nullptr, T(op->alpha), T(op->beta), T(0), nullptr, st, nullptr,
                                  S.mb[m + 1], &h->mg[m + 1].patch, h->mg[m + 1].cstride));
    const double cc = (double)xm[0] * xm[1] * xm[2] * h->ncomp;
    prof_end(st, ev, PC_RESTRICT, (2.0 * 8 + 1.0) * sizeof(T) * cc, cc * 8);
  } else {
    TRY(restrict_blocks<T, D, TR>(lv, cv, op->d_mgx[m], h->ncomp, xm, true, x, b, S.mb[m + 1], op->alpha, op->beta, st));
  }
  TRY(mg_level0<T, D, TR>(op, p, m + 1, S.mb[m + 1], S.mx[m + 1], S.mt[m + 1], st));
  TRY(prolong_blocks<T, D>(lv, cv, op->d_mgx[m], h->ncomp, xm, S.mx[m + 1], x, (T*)nullptr, st));
  TRY(smooth_from<T, D, TR>(h, 0, lv, b, x, t, p.nu2, op->alpha, op->beta, p.omega, false, st));
  return AMR_OK;
}

// ---------------------------------------------------------------- composite transpose
// S.W <- (A^comp)^T x over every covered cell (valid entries are the result; the rest is
// scratch): z = x on valid cells (0 elsewhere, copies of siblings in the copy ghosts),
// per-level transposed stencil (physical-ghost coefficients included), transposed
// refluxing, transposed AMRCFI, transposed average-down (coarse to fine).
template <typename T, int D>
amr_status composite_AT(amr_operator* op, const T* x, cudaStream_t st, int only_level = -1) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  const size_t bytes = (size_t)h->nelems * sizeof(T);
  CK(cudaMemsetAsync(S.Z, 0, bytes, st));
  CK(cudaMemsetAsync(S.W, 0, bytes, st));
  for (int l = 0; l < h->L; ++l) {
    if (only_level >= 0 && l != only_level) continue;
    LevelView lv = level_view(h, l, op->bc);
    Geo g = geo_of(lv);
    launch(k_valid_out<T, D>, g.grid, g.block, 0, st, lv, g.nby, x, (const T*)nullptr, S.Z, h->d_valid);
    TRY(launch_check());
    TRY(copy_fill<T>(h, l, S.Z, st));
  }
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, op->bc);
    TRY((level_op<T, D, true>(OP_APPLY, lv, S.Z, nullptr, S.W, nullptr, op->alpha, op->beta, 0.0, nullptr, st)));
  }
  const int nt = 128;
  for (int l = 0; l + 1 < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.nreflux == 0) continue;
    launch(k_reflux_T<T, D>, (unsigned)((dl.nreflux + nt - 1) / nt), nt, 0, st, 
        level_view(h, l, op->bc), level_view(h, l + 1, op->bc), dl.reflux, dl.nreflux, S.Z, Out3<T>{{S.W, S.W, S.W}},
        T(op->beta), 0);
    TRY(launch_check());
  }
  for (int l = 0; l < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.ncopy == 0) continue;
    launch(k_copy_T<T>, (unsigned)((dl.ncopy + nt - 1) / nt), nt, 0, st, dl.copy, dl.ncopy, S.W);
    TRY(launch_check());
  }
  for (int l = h->L - 1; l >= 1; --l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.ncfi == 0) continue;
    const LevelView fv = level_view(h, l, op->bc);
    launch(k_cfi_T<T, D>, (unsigned)((dl.ncfi + nt - 1) / nt), nt, 0, st, 
        dl.cfi, dl.ncfi, dl.cfi_side, h->lev[l - 1].d_patches, h->lev[l].d_patches, h->r, S.Z, S.W, S.W,
        T(op->beta * fv.inv12h2), T(1));
    TRY(launch_check());
  }
  for (int l = 0; l + 1 < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.nxfer == 0) continue;
    const int fy = 2 * dl.xfer_max[1];
    const int nby = (fy + BY - 1) / BY;
    dim3 grid((2 * dl.xfer_max[0] + BX - 1) / BX, nby * (D == 3 ? 2 * dl.xfer_max[2] : 1), dl.nxfer);
    launch(k_avgdown_T<T, D>, grid, dim3(BX, BY, 1), 0, st, level_view(h, l + 1, nullptr), level_view(h, l, nullptr), dl.xfer,
                                                      S.W, nby);
    TRY(launch_check());
  }
  return AMR_OK;
}

// out = f - S.W on the valid cells of level l (the other cells of out are left alone);
// l < 0: every level, invalid cells set to zero.
template <typename T, int D>
amr_status transpose_residual(amr_operator* op, int l, const T* f, T* out, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  for (int m = 0; m < h->L; ++m) {
    if (l >= 0 && m != l) continue;
    LevelView lv = level_view(h, m, nullptr);
    Geo g = geo_of(lv);
    if (l < 0) {
      launch(k_valid_out<T, D>, g.grid, g.block, 0, st, lv, g.nby, S.W, f, out, h->d_valid);
    } else {
      // valid cells only: residual, invalid cells untouched
      launch(k_level_op_masked_copy<T, D>, g.grid, g.block, 0, st, lv, g.nby, S.W, f, out, h->d_valid);
    }
    TRY(launch_check());
  }
  return AMR_OK;
}

template <typename T, int D>
Geo xfer_geo(const DeviceLists& dl, bool fine_cells, int& nby) {
  Geo g;
  const int fy = (fine_cells ? 2 : 1) * dl.xfer_max[1];
  nby = (fy + BY - 1) / BY;
  g.nby = nby;
  g.grid = dim3(((fine_cells ? 2 : 1) * dl.xfer_max[0] + BX - 1) / BX,
                nby * (D == 3 ? (fine_cells ? 2 : 1) * dl.xfer_max[2] : 1), dl.nxfer);
  return g;
}

// Adjoint V-cycle: the exact transpose of vcycle_corr's AMR part (the forward program run
// backwards, every step transposed; the transpose of weighted-Jacobi sweeps from zero on A
// is the same number of sweeps from zero on A^T), with a V-cycle on A^T for all of level
// 0.  Input: r (valid cells); output S.X = M^T r where M is the forward V-cycle's AMR part.
template <typename T, int D>
amr_status vcycle_corr_T(amr_operator* op, const amr_solver_params& p, const T* r, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  const int L = h->L - 1;
  const size_t bytes = (size_t)h->nelems * sizeof(T);
  // adjoint buffers: Xb = S.X (adjoint of X), Eb = S.E, Rb = S.R, rb = S.rin (output), tmp = S.Y
  T* Xb = S.X;
  T* Eb = S.E;
  T* Rb = S.R;
  T* rb = S.rin;
  T* tmp = S.Y;
  if (r == rb) {
    CK(cudaMemcpyAsync(S.Y, r, bytes, cudaMemcpyDeviceToDevice, st));  // mixed precision: input lives in rin
    r = S.Y;
  }
  CK(cudaMemsetAsync(Xb, 0, bytes, st));
  std::vector<LevelView> lv(h->L);
  for (int l = 0; l <= L; ++l) lv[l] = level_view(h, l, op->bc);
  for (int l = 0; l <= L; ++l) {
    Geo g = geo_of(lv[l]);
    launch(k_axpy_valid<T, D>, g.grid, g.block, 0, st, lv[l], g.nby, r, Xb, T(1), h->d_valid);
    TRY(launch_check());
  }
  CK(cudaMemsetAsync(Eb, 0, bytes, st));
  CK(cudaMemsetAsync(Rb, 0, bytes, st));
  CK(cudaMemsetAsync(rb, 0, bytes, st));
  CK(cudaMemsetAsync(S.T1, 0, bytes, st));
  CK(cudaMemsetAsync(S.T2, 0, bytes, st));
  const double a_ = op->alpha, b_ = op->beta;
  const int nt = 128;
  // ---- reverse of the up-leg, finest level first
  for (int l = L; l >= 1; --l) {
    const DeviceLists& cl = h->lev[l - 1].dev;
    // U4^T: delta_bar = Eb_l + Xb_l (into tmp, level l)
    CK(cudaMemsetAsync(tmp, 0, bytes, st));
    TRY((axpy<T, T, D>(lv[l], Eb, tmp, (T*)nullptr, 1.0, st)));
    TRY((axpy<T, T, D>(lv[l], Xb, tmp, (T*)nullptr, 1.0, st)));
    // U3^T: Rb_l += S'^T delta_bar (nu2 sweeps from zero on A_l^T)
    TRY((smooth_from_zero<T, D, true>(h, l, lv[l], tmp, S.T1, S.T2, p.nu2, a_, b_, p.omega, true, st)));
    TRY((axpy<T, T, D>(lv[l], S.T1, Rb, (T*)nullptr, 1.0, st)));
    // U2^T: Eb_l -= A_l^T Rb_l ; Eb_{l-1} -= A_fc^T Rb_l
    TRY(copy_fill<T>(h, l, Rb, st));
    TRY((level_op<T, D, true>(OP_RESID, lv[l], Rb, Eb, Eb, nullptr, a_, b_, 0.0, nullptr, st)));
    {
      const DeviceLists& dl = h->lev[l].dev;
      if (dl.ncfi) {
        launch(k_cfi_T<T, D>, (unsigned)((dl.ncfi + nt - 1) / nt), nt, 0, st, 
            dl.cfi, dl.ncfi, dl.cfi_side, h->lev[l - 1].d_patches, h->lev[l].d_patches, h->r, Rb, (const T*)nullptr,
            Eb, T(b_ * lv[l].inv12h2), T(-1));
        TRY(launch_check());
      }
    }
    // U1^T: Eb_{l-1} += P^T (Eb_l + Xb_l)
    if (cl.nxfer) {
      int nby;
      Geo g = xfer_geo<T, D>(cl, true, nby);
      launch(k_prolong_T<T, D>, g.grid, dim3(BX, BY, 1), 0, st, lv[l], lv[l - 1], cl.xfer, Eb, Xb, Eb, nby);
      TRY(launch_check());
    }
    // the forward prolongation read sibling values through copy ghosts of level l-1
    if (cl.ncopy) {
      launch(k_copy_T<T>, (unsigned)((cl.ncopy + nt - 1) / nt), nt, 0, st, cl.copy, cl.ncopy, Eb);
      TRY(launch_check());
    }
  }
  // ---- level 0: Eb_0 += Xb_0 ; Rb_0 += MG0^T(Eb_0)
  TRY((axpy<T, T, D>(lv[0], Xb, Eb, (T*)nullptr, 1.0, st)));
  CK(cudaMemsetAsync(tmp, 0, bytes, st));
  TRY((mg_level0<T, D, true>(op, p, 0, Eb, tmp, S.T1, st)));
  TRY((axpy<T, T, D>(lv[0], tmp, Rb, (T*)nullptr, 1.0, st)));
  // ---- reverse of the down-leg, coarsest level first
  for (int l = 1; l <= L; ++l) {
    const DeviceLists& cl = h->lev[l - 1].dev;
    // D4^T: rb_{l-1} += Rb_{l-1} (valid) ; Xb -= valid part of A^T (Rb_{l-1} on level l-1 valid cells)
    {
      Geo g = geo_of(lv[l - 1]);
      launch(k_axpy_valid<T, D>, g.grid, g.block, 0, st, lv[l - 1], g.nby, Rb, rb, T(1), h->d_valid);
      TRY(launch_check());
    }
    TRY((composite_AT<T, D>(op, Rb, st, l - 1)));
    for (int m = l; m <= L; ++m) {
      Geo g = geo_of(lv[m]);
      launch(k_axpy_valid<T, D>, g.grid, g.block, 0, st, lv[m], g.nby, S.W, Xb, T(-1), h->d_valid);
      TRY(launch_check());
    }
    // D3^T: tmp_l = Avg^T (Rb_{l-1} on invalid cells) ; Rb_l += tmp_l ; Eb_l -= A_l^T tmp_l
    CK(cudaMemsetAsync(tmp, 0, bytes, st));
    if (cl.nxfer) {
      int nby;
      Geo g = xfer_geo<T, D>(cl, true, nby);
      launch(k_avgdown_T2<T, D>, g.grid, dim3(BX, BY, 1), 0, st, lv[l], lv[l - 1], cl.xfer, Rb, tmp, nby);
      TRY(launch_check());
    }
    TRY((axpy<T, T, D>(lv[l], tmp, Rb, (T*)nullptr, 1.0, st)));
    TRY(copy_fill<T>(h, l, tmp, st));
    TRY((level_op<T, D, true>(OP_RESID, lv[l], tmp, Eb, Eb, nullptr, a_, b_, 0.0, nullptr, st)));
    // D2^T: Eb_l += Xb_l
    TRY((axpy<T, T, D>(lv[l], Xb, Eb, (T*)nullptr, 1.0, st)));
    // D1^T: Rb_l += S^T Eb_l
    TRY((smooth_from_zero<T, D, true>(h, l, lv[l], Eb, S.T1, S.T2, p.nu1, a_, b_, p.omega, true, st)));
    TRY((axpy<T, T, D>(lv[l], S.T1, Rb, (T*)nullptr, 1.0, st)));
  }
  // R_L = r_L: rb_L += Rb_L (valid cells)
  {
    Geo g = geo_of(lv[L]);
    launch(k_axpy_valid<T, D>, g.grid, g.block, 0, st, lv[L], g.nby, Rb, rb, T(1), h->d_valid);
    TRY(launch_check());
  }
  CK(cudaMemcpyAsync(S.X, rb, bytes, cudaMemcpyDeviceToDevice, st));
  return AMR_OK;
}

// ---------------------------------------------------------------- composite V-cycle
// Correction form: given the composite residual r (covered cells), S.X receives the
// V-cycle's approximation of A^{-1} r (homogeneous data).
// Whether AMR level l's smoothing runs as temporally blocked launches: FP32 forward V-cycles
// in 2-D, a single box, whose coarsened cells lie in one coarse box, sweep counts within
// the halo budget, and a box small enough for the region table.
template <typename T, int D>
bool blocked_amr_level(const amr_operator* op, const amr_solver_params& p, int l) {
  if (D != 2 || sizeof(T) != 4 || !p.temporal_blocking) return false;
  if (p.nu1 < 1 || p.nu1 > BLK_MAX_NU || p.nu2 > BLK_MAX_NU) return false;
  const amr_hierarchy* h = op->h;
  if (h->lev[l].patches.size() != 1 || h->lev[l - 1].xfer.size() != 1) return false;
  const PatchDesc& fp = h->lev[l].patches[0];
  const XferBlock& xb = h->lev[l - 1].xfer[0];
  for (int d = 0; d < 2; ++d)
    if (xb.clo[d] * 2 != fp.lo[d] || (xb.chi[d] + 1) * 2 != fp.lo[d] + fp.n[d]) return false;
  return true;
}

template <typename T, int D>
amr_status vcycle_corr(amr_operator* op, const amr_solver_params& p, const T* r, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  Scratch<T>& S = scratch<T>(op);
  const int L = h->L - 1;
  const size_t bytes = (size_t)h->nelems * sizeof(T);
  CK(cudaMemsetAsync(S.E, 0, bytes, st));
  CK(cudaMemsetAsync(S.X, 0, bytes, st));
  CK(cudaMemsetAsync(S.T1, 0, bytes, st));
  CK(cudaMemsetAsync(S.T2, 0, bytes, st));
  for (int c = 0; c < h->ncomp; ++c) {
    long long a, b;
    level_range(h, L, a, b, c);
    CK(cudaMemcpyAsync(S.R + a, r + a, (size_t)(b - a) * sizeof(T), cudaMemcpyDeviceToDevice, st));
  }
  std::vector<LevelView> lv(h->L);
  for (int l = 0; l <= L; ++l) lv[l] = level_view(h, l, op->bc);
  const double a_ = op->alpha, b_ = op->beta;
  // ---- down
  for (int l = L; l >= 1; --l) {
    const DeviceLists& cl = h->lev[l - 1].dev;
    bool deferred = false;
    if (blocked_amr_level<T, D>(op, p, l)) {
      // one launch: nu1 sweeps from zero (zero CF ghosts) into E_l, X_l += E_l, and the
      // mean of the fine residual R_l - A_l E_l into R_{l-1} on the covered cells
      const PatchDesc& fp = h->lev[l].patches[0];
      const PatchDesc& cpd = h->lev[l - 1].patches[h->lev[l - 1].xfer[0].cpatch];
      const int tt = blk_tile(fp.n), hd = 2 * p.nu1 + 2;
      const T ood = T(p.omega / (a_ - 60.0 * b_ * lv[l].inv12h2));
      dim3 grid((fp.n[0] + tt - 1) / tt, (fp.n[1] + tt - 1) / tt, 1);
      cudaEvent_t ev;
      prof_begin(st, &ev);
      launch_down2d<T>(tt, p.nu1, grid, blk_smem_fx<T>(fp.n, p.nu1, true), st, lv[l], fp, cpd, tt, tt, hd, p.nu1,
                       (const T*)S.R, S.E, S.X, S.R, T(a_), T(b_), T(p.omega), ood);
      TRY(launch_check());
      prof_end(st, ev, PC_DOWN, (3.0 + 0.25) * sizeof(T) * (double)fp.n[0] * fp.n[1]);  // f in; e, x, coarse f out
    } else {
      TRY(smooth_from_zero<T, D>(h, l, lv[l], S.R, S.E, S.T1, p.nu1, a_, b_, p.omega, true, st));
      TRY(axpy<T, T, D>(lv[l], S.E, S.X, (T*)nullptr, 1.0, st));
      TRY(copy_fill<T>(h, l, S.E, st));
      deferred = true;  // the fine residual's mean is restricted after the level-(l-1) residual
    }
    // valid cells of level l-1: composite residual r - A^comp X
    for (int m = l - 1; m >= 0; --m) {
      const DeviceLists& dm = h->lev[m].dev;
      TRY(restrict_blocks<T, D>(lv[m + 1], lv[m], dm.xfer, dm.nxfer, dm.xfer_max, false, S.X, (const T*)nullptr, S.X,
                                0.0, 0.0, st));
    }
    if (l - 1 >= 1) TRY(cfi_fill<T, D>(h, l - 1, S.X, S.X, false, st));
    TRY(copy_fill<T>(h, l - 1, S.X, st));
    TRY(cfi_fill<T, D>(h, l, S.X, S.X, false, st));
    TRY(copy_fill<T>(h, l, S.X, st));
    if (deferred) {
      // every cell of level l-1, then its invalid cells overwritten by the mean of the fine
      // residual R_l - A_l E_l (zero CF ghosts): the same values as the masked residual
      // after the restriction, without the mask (the restriction reads neither array the
      // level-(l-1) residual writes)
      TRY(level_op<T, D>(OP_RESID, lv[l - 1], S.X, r, S.R, nullptr, a_, b_, 0.0, nullptr, st));
      if (D == 3 && lv[l - 1].npatch == lv[l - 1].ncomp && sw_eligible(lv[l]) && lv[l].maxn[2] % 2 == 0 &&
          tile_rows_for(lv[l], sizeof(T)) == TILE_BULK) {
        // a single-patch fine level over a single-patch coarse level: the bulk-copy
        // restriction (the arithmetic of k_restrict)
        cudaEvent_t ev;
        prof_begin(st, &ev);
        TRY((launch_sw<T, OP_RESTRICT>(lv[l], S.E, S.R, (T*)nullptr, T(a_), T(b_), T(0), nullptr, st, nullptr, S.R,
                                       &lv[l - 1].p0, lv[l - 1].cstride)));
        const double cc = lv[l].ncells / 8.0;
        prof_end(st, ev, PC_RESTRICT, (2.0 * 8 + 1.0) * sizeof(T) * cc, cc * 8);
      } else {
        TRY(restrict_blocks<T, D>(lv[l], lv[l - 1], cl.xfer, cl.nxfer, cl.xfer_max, true, S.E, S.R, S.R, a_, b_, st));
      }
    } else {
      TRY(level_op<T, D>(OP_RESID, lv[l - 1], S.X, r, S.R, nullptr, a_, b_, 0.0, h->d_valid, st));
    }
    P3<T> xc{{S.X, S.X, S.X}}, xf{{S.X, S.X, S.X}}, nb{{nullptr, nullptr, nullptr}};
    TRY(reflux<T, D>(h, l - 1, lv[l - 1], lv[l], xc, xf, nb, S.R, -b_, 0, st));
  }
  // ---- level 0: single-level V-cycle on all of level 0
  TRY(mg_level0<T, D>(op, p, 0, S.R, S.E, S.T1, st));
  TRY(axpy<T, T, D>(lv[0], S.E, S.X, (T*)nullptr, 1.0, st));
  // ---- up
  for (int l = 1; l <= L; ++l) {
    const DeviceLists& cl = h->lev[l - 1].dev;
    TRY(copy_fill<T>(h, l - 1, S.E, st));
    TRY(prolong_blocks<T, D>(lv[l], lv[l - 1], cl.xfer, cl.nxfer, cl.xfer_max, S.E, S.E, S.X, st));
    TRY(cfi_fill<T, D>(h, l, S.E, S.E, false, st));
    TRY(copy_fill<T>(h, l, S.E, st));
    TRY(level_op<T, D>(OP_RESID, lv[l], S.E, S.R, S.R, nullptr, a_, b_, 0.0, nullptr, st));
    if (blocked_amr_level<T, D>(op, p, l) && p.nu2 >= 1) {
      // one launch: nu2 sweeps from zero on R_l (zero CF ghosts), added to E_l and X_l
      const PatchDesc& fp = h->lev[l].patches[0];
      const int tt = blk_tile(fp.n), hu = 2 * p.nu2;
      const T ood = T(p.omega / (a_ - 60.0 * b_ * lv[l].inv12h2));
      dim3 grid((fp.n[0] + tt - 1) / tt, (fp.n[1] + tt - 1) / tt, 1);
      cudaEvent_t ev;
      prof_begin(st, &ev);
      launch_post2d<T>(tt, p.nu2, grid, blk_smem_fx<T>(fp.n, p.nu2, false), st, lv[l], fp, tt, tt, hu, p.nu2,
                       (const T*)S.R, S.E, S.X, T(a_), T(b_), T(p.omega), ood);
      TRY(launch_check());
      prof_end(st, ev, PC_UP, 5.0 * sizeof(T) * (double)fp.n[0] * fp.n[1]);  // r in; e, x read and written
    } else {
      TRY(smooth_from_zero<T, D>(h, l, lv[l], S.R, S.T1, S.T2, p.nu2, a_, b_, p.omega, true, st));
      TRY(axpy<T, T, D>(lv[l], S.T1, S.E, S.X, 1.0, st));
    }
  }
  return AMR_OK;
}

// ---------------------------------------------------------------- composite pieces
// (FP64 in the refinement loop and the projection; FP32 for the inner residual of the
// mixed-precision correction, see mixed_correction)
template <int D, typename T>
amr_status avgdown_all(amr_hierarchy* h, T* x, cudaStream_t st) {
  for (int m = h->L - 2; m >= 0; --m) {
    const DeviceLists& dm = h->lev[m].dev;
    LevelView f = level_view(h, m + 1, nullptr), c = level_view(h, m, nullptr);
    TRY(restrict_blocks<T, D>(f, c, dm.xfer, dm.nxfer, dm.xfer_max, false, x, (const T*)nullptr, x, 0.0, 0.0, st));
  }
  return AMR_OK;
}

template <int D, typename T>
amr_status fill_ghosts_all(amr_hierarchy* h, T* x, cudaStream_t st) {
  TRY(avgdown_all<D>(h, x, st));
  for (int l = 0; l < h->L; ++l) {
    if (l >= 1) TRY((cfi_fill<T, D>(h, l, x, x, false, st)));
    TRY(copy_fill<T>(h, l, x, st));
  }
  return AMR_OK;
}

// out = A^comp x (mode OP_APPLY) or out = f - A^comp x (OP_RESID); covered cells.
template <int D, typename T>
amr_status composite_op(amr_operator* op, int mode, T* x, const T* f, T* out, const T* bc, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  TRY(fill_ghosts_all<D>(h, x, st));
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, op->bc);
    TRY((level_op<T, D>(mode, lv, x, f, out, bc, op->alpha, op->beta, 0.0, nullptr, st)));
  }
  for (int l = h->L - 2; l >= 0; --l) {
    LevelView c = level_view(h, l, op->bc), fv = level_view(h, l + 1, op->bc);
    P3<T> xc{{x, x, x}}, xf{{x, x, x}}, nb{{bc, bc, bc}};
    TRY((reflux<T, D>(h, l, c, fv, xc, xf, nb, out, mode == OP_APPLY ? op->beta : -op->beta, 0, st)));
  }
  TRY(avgdown_all<D>(h, out, st));  // COH-4
  return AMR_OK;
}

template <typename T, int D>
amr_status maxnorm(amr_hierarchy* h, const T* x, bool use_mask, double* out_host, cudaStream_t st) {
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(h->d_scalar);
  CK(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st));
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    Geo g = geo_of(lv);
    launch(k_maxnorm<T, D>, g.grid, g.block, 0, st, lv, g.nby, x, use_mask ? h->d_valid : nullptr, acc);
    TRY(launch_check());
  }
  CK(cudaMemcpyAsync(h->h_scalar, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *out_host = h->h_scalar[0];
  return AMR_OK;
}

// Blocks of the grid-stride weighted sum of one level (k_wsum_gs): one per 256 cells, at
// most 512; the partials are added in this fixed order, so a given hierarchy always gets
// the same rounding.
inline long long wsum_blocks(const LevelView& lv) {
  return std::min<long long>(512, std::max<long long>(1, ((long long)lv.ncells + 255) / 256));
}

// The weighted sums keep one partial per block in the hierarchy's 8192-slot scratch: a
// hierarchy that needs more is rejected before anything is launched.
inline amr_status wsum_fits(amr_hierarchy* h) {
  long long nb = 0;
  for (int l = 0; l < h->L; ++l) nb += wsum_blocks(level_view(h, l, nullptr));
  if (nb > 8192) {
    set_error("reduction scratch too small: the hierarchy needs " + std::to_string(nb) + " reduction blocks (8192 max)");
    return AMR_ERR_INVALID_ARG;
  }
  return AMR_OK;
}

// d_out[0] = sum over valid cells of h^D x (compensated); d_out[1] = boundary flux sum
template <int D>
amr_status wsum(amr_hierarchy* h, const double* x, const double* bc, const int* bc_types, double* d_out,
                cudaStream_t st, bool unweighted = false) {
  long long base = 0;
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    const long long nb = wsum_blocks(lv);
    if (base + nb > 8192) {
      set_error("reduction scratch too small");
      return AMR_ERR_INVALID_ARG;
    }
    launch(k_wsum_gs<D>, (unsigned)nb, 256, 0, st, lv, x, h->d_valid, unweighted ? 1.0 : std::pow(lv.h, D), h->d_red, base);
    TRY(launch_check());
    base += nb;
  }
  launch(k_dd_final, 1, 256, 0, st, h->d_red, base, d_out);
  TRY(launch_check());
  if (bc != nullptr && bc_types != nullptr) {
    long long bb = 0;
    for (int l = 0; l < h->L; ++l) {
      LevelView lv = level_view(h, l, bc_types);
      const int nblk = lv.npatch * 2 * D;
      launch(k_bsum<D>, nblk, 256, 0, st, lv, bc, h->d_valid, std::pow(lv.h, D - 1), h->d_red, bb);
      TRY(launch_check());
      bb += nblk;
    }
    launch(k_dd_final, 1, 256, 0, st, h->d_red, bb, d_out + 1);
    TRY(launch_check());
  } else {
    CK(cudaMemsetAsync(d_out + 1, 0, sizeof(double), st));
  }
  return AMR_OK;
}

double valid_volume(const amr_hierarchy* h) {
  // number of valid cells per level times h^D (exact small integers times powers of 2)
  long double v = 0.0L;
  size_t q = 0;
  for (int l = 0; l < h->L; ++l) {
    long long cnt = 0;
    for (const PatchDesc& p : h->lev[l].patches) {
      const long long nc = (long long)p.n[0] * p.n[1] * p.n[2];
      for (long long i = 0; i < nc; ++i) cnt += h->im_valid[q + i];
      q += nc;
    }
    v += (long double)cnt * std::pow((long double)h->lev[l].h, (long double)h->D);
  }
  return (double)v;
}

template <int D>
amr_status shift_all(amr_hierarchy* h, double* x, const double* d_m, bool valid_only, double sign, cudaStream_t st) {
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    Geo g = geo_of(lv);
    launch(k_shift<D>, g.grid, g.block, 0, st, lv, g.nby, x, d_m, valid_only ? h->d_valid : nullptr, sign);
    TRY(launch_check());
  }
  return AMR_OK;
}

template <int D>
amr_status solvability_fix_impl(amr_operator* op, double* f, const double* bc, double* m_host, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  TRY(wsum_fits(h));
  TRY(wsum<D>(h, f, bc, op->bc, h->d_scalar + 2, st));
  launch(k_mean_from_sums, 1, 1, 0, st, h->d_scalar + 2, h->d_scalar + 3, op->beta, valid_volume(h), h->d_scalar + 4);
  TRY(launch_check());
  TRY(shift_all<D>(h, f, h->d_scalar + 4, true, -1.0, st));
  if (m_host) {
    CK(cudaMemcpyAsync(h->h_scalar + 4, h->d_scalar + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *m_host = h->h_scalar[4];
  }
  return AMR_OK;
}

template <int D>
amr_status mean_zero_impl(amr_hierarchy* h, double* x, double* mean_host, cudaStream_t st) {
  TRY(wsum_fits(h));
  TRY(avgdown_all<D>(h, x, st));
  TRY(wsum<D>(h, x, nullptr, nullptr, h->d_scalar + 2, st));
  launch(k_mean_from_sums, 1, 1, 0, st, h->d_scalar + 2, nullptr, 0.0, valid_volume(h), h->d_scalar + 4);
  TRY(launch_check());
  TRY(shift_all<D>(h, x, h->d_scalar + 4, false, -1.0, st));
  if (mean_host) {
    CK(cudaMemcpyAsync(h->h_scalar + 4, h->d_scalar + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *mean_host = h->h_scalar[4];
  }
  return AMR_OK;
}

// Transpose of the pure-Neumann projector F = I - 1 w^T/(w^T 1) (w = h^D on valid cells; F
// is both the solvability correction of Sec. 6.4 with homogeneous data and the mean-zero
// step): x <- x - w (1^T x)/(1^T w) on the valid cells.
template <int D>
amr_status neumann_fix_T(amr_hierarchy* h, double* x, double* m_host, cudaStream_t st) {
  TRY(wsum_fits(h));
  TRY(wsum<D>(h, x, nullptr, nullptr, h->d_scalar + 2, st, true));
  launch(k_mean_from_sums, 1, 1, 0, st, h->d_scalar + 2, nullptr, 0.0, valid_volume(h), h->d_scalar + 4);
  TRY(launch_check());
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    Geo g = geo_of(lv);
    launch(k_shift<D>, g.grid, g.block, 0, st, lv, g.nby, x, h->d_scalar + 4, h->d_valid, -std::pow(lv.h, D));
    TRY(launch_check());
  }
  if (m_host) {
    CK(cudaMemcpyAsync(h->h_scalar + 4, h->d_scalar + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *m_host = h->h_scalar[4];
  }
  return AMR_OK;
}

// max-norm over valid cells into *out (IEEE bits, atomicMax); no host readback
template <typename T, int D>
amr_status maxnorm_dev(amr_hierarchy* h, const T* x, unsigned long long* out, cudaStream_t st) {
  CK(cudaMemsetAsync(out, 0, sizeof(unsigned long long), st));
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    Geo g = geo_of(lv);
    launch(k_maxnorm<T, D>, g.grid, g.block, 0, st, lv, g.nby, x, h->d_valid, out);
    TRY(launch_check());
  }
  return AMR_OK;
}

// Bounded wait of about ``ns`` nanoseconds (at most 2^20 polls of the global timer).
__global__ void k_headstart(unsigned long long ns) {
  pdl_wait();
  if (threadIdx.x != 0) return;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < (1 << 20); ++it) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 >= ns) break;
    __nanosleep(500);
  }
}

// Stopping test of Sec. 7 on the device: records the residual norm, decides whether the
// while-loop of the captured solve runs another V-cycle.
__global__ void k_check(cudaGraphConditionalHandle handle, int use_cond, const unsigned long long* __restrict__ rbits,
                        const unsigned long long* __restrict__ fbits, double rtol, double atol, int maxv,
                        DevStats* __restrict__ s) {
  pdl_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r = __longlong_as_double((long long)*rbits);
  const double fn = __longlong_as_double((long long)*fbits);
  const int it = s->iter;
  if (it < 64) s->hist[it] = r;
  const double tol = fmax(rtol * fn, atol);
  unsigned int cont = 0;
  if (!isfinite(r)) s->status = 2;
  else if (r <= tol) s->status = 0;
  else if (it >= maxv) s->status = 1;
  else {
    cont = 1;
    s->iter = it + 1;
  }
  if (use_cond) cudaGraphSetConditional(handle, cont);
}

// ---------------------------------------------------------------- mixed-precision correction
// cycles_per_refinement (mixed precision only; 1 otherwise) and the cap on refinement steps
inline int cpr_of(const amr_solver_params& p) { return p.precision == AMR_MIXED ? p.cycles_per_refinement : 1; }
inline int max_steps(const amr_solver_params& p) { return (p.max_vcycles + cpr_of(p) - 1) / cpr_of(p); }

// the two buffers of the later correction cycles; allocated by the solve entry points before
// any stream capture begins (allocation is not allowed inside a capture)
amr_status ensure_inner(amr_operator* op) {
  if (op->inner_x != nullptr && op->inner_r != nullptr) return AMR_OK;
  const size_t bytes = (size_t)op->h->nelems * sizeof(float);
  float* a = nullptr;
  float* b = nullptr;
  if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess ||
      cudaMemset(a, 0, bytes) != cudaSuccess || cudaMemset(b, 0, bytes) != cudaSuccess) {
    cudaFree(a);
    cudaFree(b);
    cudaGetLastError();
    set_error("allocation of the correction-cycle buffers failed");
    return AMR_ERR_CUDA;
  }
  cudaFree(op->inner_x);
  cudaFree(op->inner_r);
  op->inner_x = a;
  op->inner_r = b;
  return AMR_OK;
}

// The FP32 correction of one refinement step into s32.X from the FP32 residual s32.rin:
// one composite V-cycle, then (cycles_per_refinement > 1) further cycles on the FP32
// composite residual rin - A X of the correction so far (homogeneous boundary data), each
// added to it.  The correction so far moves to inner_x and the next cycle writes the other
// buffer, so no copy is made.
template <int D>
amr_status mixed_correction(amr_operator* op, const amr_solver_params& p, cudaStream_t st) {
  Scratch<float>& S = op->s32;
  TRY((vcycle_corr<float, D>(op, p, S.rin, st)));
  if (cpr_of(p) <= 1) return AMR_OK;
  if (op->inner_x == nullptr || op->inner_r == nullptr) {
    set_error("correction-cycle buffers were not allocated before the solve");
    return AMR_ERR_INVALID_ARG;
  }
  amr_hierarchy* h = op->h;
  for (int c = 1; c < cpr_of(p); ++c) {
    std::swap(S.X, op->inner_x);
    TRY(composite_op<D>(op, OP_RESID, op->inner_x, (const float*)S.rin, op->inner_r, (const float*)nullptr, st));
    TRY((vcycle_corr<float, D>(op, p, op->inner_r, st)));
    for (int l = 0; l < h->L; ++l)
      TRY((axpy<float, float, D>(level_view(h, l, nullptr), op->inner_x, S.X, (float*)nullptr, 1.0, st)));
  }
  return AMR_OK;
}

// ---------------------------------------------------------------- solve
template <int D>
amr_status solve_graph(amr_operator* op, const amr_solver_params& p, double* phi, const double* f, const double* bc,
                       amr_solve_stats* stats, cudaStream_t st);

template <int D>
amr_status solve_impl(amr_operator* op, const amr_solver_params& p, double* phi, const double* f, const double* bc,
                      amr_solve_stats* stats, cudaStream_t st) {
  // instrumented runs use the host-driven loop (event records cannot sit in graph bodies)
  if (p.use_graph && !g_prof.on) return solve_graph<D>(op, p, phi, f, bc, stats, st);
  amr_hierarchy* h = op->h;
  const size_t bytes = (size_t)h->nelems * sizeof(double);
  amr_solve_stats loc{};
  CK(cudaMemcpyAsync(op->F, f, bytes, cudaMemcpyDeviceToDevice, st));
  if (op->neumann) TRY(solvability_fix_impl<D>(op, op->F, bc, &loc.removed_mean, st));
  if (p.zero_initial) CK(cudaMemsetAsync(phi, 0, bytes, st));
  TRY(avgdown_all<D>(h, op->F, st));
  double fn = 0.0;
  TRY(maxnorm<double, D>(h, op->F, true, &fn, st));
  loc.rhs_norm = fn;
  const double tol = std::max(p.rtol * fn, p.atol);
  if (p.precision == AMR_MIXED) TRY(ensure_scratch<float>(op));
  if (cpr_of(p) > 1) TRY(ensure_inner(op));
  else TRY(ensure_scratch<double>(op));
  amr_status result = AMR_ERR_NOT_CONVERGED;
  double res = 0.0;
  int it = 0;
  for (;; ++it) {
    TRY(composite_op<D>(op, OP_RESID, phi, op->F, op->Res, bc, st));
    TRY(maxnorm<double, D>(h, op->Res, true, &res, st));
    if (it < 64) loc.res_history[it] = res;
    if (!std::isfinite(res)) { result = AMR_ERR_NONFINITE; set_error("residual is not finite"); break; }
    if (res <= tol) { result = AMR_OK; break; }
    if (it >= max_steps(p)) { set_error("max_vcycles reached"); break; }
    if (g_prof.on) {
      // instrumented run: keep the GPU busy for a moment so that the host queues this
      // V-cycle's launches ahead of execution and the event intervals hold kernels only
      launch(k_headstart, 1, 32, 0, st, 1500000ull);
      TRY(launch_check());
    }
    if (p.precision == AMR_MIXED) {
      Scratch<float>& S = op->s32;
      for (int l = 0; l < h->L; ++l) TRY(convert<double, float, D>(level_view(h, l, nullptr), op->Res, S.rin, st));
      TRY(mixed_correction<D>(op, p, st));
      for (int l = 0; l < h->L; ++l) TRY(axpy<float, double, D>(level_view(h, l, nullptr), S.X, phi, (double*)nullptr, 1.0, st));
    } else {
      Scratch<double>& S = op->s64;
      TRY(vcycle_corr<double, D>(op, p, op->Res, st));
      for (int l = 0; l < h->L; ++l) TRY(axpy<double, double, D>(level_view(h, l, nullptr), S.X, phi, (double*)nullptr, 1.0, st));
    }
  }
  loc.vcycles = it * (p.precision == AMR_MIXED ? cpr_of(p) : 1);
  loc.final_res = res;
  if (op->neumann && result == AMR_OK) TRY(mean_zero_impl<D>(h, phi, nullptr, st));
  else TRY(avgdown_all<D>(h, phi, st));
  if (stats) *stats = loc;
  return result;
}

// One V-cycle iteration of the solve loop (V-cycle on op->Res, phi += correction, new
// residual and its norm), all stream-ordered on st; used inside the captured while-body.
// grid of the whole-array passes: grid-stride, a few blocks per SM
// grid-stride element-wise kernels: one block per 256 elements, at most 8 per SM
inline unsigned flat_blocks(long long n) {
  static int nsm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int m = (dev >= 0 && dev < 64) ? nsm[dev] : 0;
  if (m == 0) {
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    m = std::max(1, m);
    if (dev >= 0 && dev < 64) nsm[dev] = m;
  }
  return (unsigned)std::min<long long>((n + 255) / 256, 8LL * m);
}

// elements of one replica of a stacked component batch (the whole array otherwise)
inline long long rep_elems(const amr_hierarchy* h) { return h->ncomp > 1 ? h->cstride : h->nelems; }

// valid-cell max-norm of x into acc[c] for every replica c, and (rin given) x rounded to FP32
inline amr_status norm_convert_field(amr_operator* op, const double* x, float* rin, unsigned long long* acc,
                                     cudaStream_t st) {
  amr_hierarchy* h = op->h;
  const long long n = rep_elems(h);
  launch(k_norm_convert, dim3(flat_blocks(n), h->ncomp, 1), 256, 0, st, n, x, (const unsigned char*)h->d_valid, rin,
         acc);
  return launch_check();
}

// valid-cell max-norm of op->Res into acc (per replica), and (mixed precision) its FP32 copy
inline amr_status norm_convert(amr_operator* op, int prec, unsigned long long* acc, cudaStream_t st) {
  return norm_convert_field(op, op->Res, prec == AMR_MIXED ? op->s32.rin : nullptr, acc, st);
}

// One V-cycle iteration of the captured solve loop: V-cycle on the residual (FP32 copy made
// by the previous norm pass in mixed precision), phi += correction on the valid cells, new
// composite residual, its norm (and FP32 copy), all stream-ordered on st.
template <int D>
amr_status iteration_body(amr_operator* op, int prec, const amr_solver_params& p, double* phi, const double* bc,
                          cudaStream_t st) {
  amr_hierarchy* h = op->h;
  unsigned long long* rbits = h->d_cnorm;
  const long long n = rep_elems(h);
  const dim3 grid(flat_blocks(n), h->ncomp, 1);
  const int* active = h->ncomp > 1 ? op->d_active : nullptr;  // converged replicas keep their phi
  if (prec == AMR_MIXED) {
    Scratch<float>& Sf = op->s32;
    TRY(mixed_correction<D>(op, p, st));
    launch(k_update_valid<float>, grid, 256, 0, st, n, (const float*)Sf.X, phi, (const unsigned char*)h->d_valid, rbits,
           active);
  } else {
    Scratch<double>& Sd = op->s64;
    TRY(vcycle_corr<double, D>(op, p, op->Res, st));
    launch(k_update_valid<double>, grid, 256, 0, st, n, (const double*)Sd.X, phi, (const unsigned char*)h->d_valid,
           rbits, active);
  }
  TRY(launch_check());
  TRY(composite_op<D>(op, OP_RESID, phi, op->F, op->Res, bc, st));
  return norm_convert(op, prec, rbits, st);
}

__global__ void k_check_b(cudaGraphConditionalHandle handle, int use_cond, int n, const unsigned long long* __restrict__ rbits,
                          const unsigned long long* __restrict__ fbits, double rtol, double atol, int maxv,
                          DevStats* __restrict__ s, int* __restrict__ active);

template <int D>
amr_status build_solve_graph(amr_operator* op, const amr_solver_params& p, double* phi, const double* bc) {
  amr_hierarchy* h = op->h;
  if (op->exec) { cudaGraphExecDestroy(op->exec); op->exec = nullptr; }
  if (op->graph) { cudaGraphDestroy(op->graph); op->graph = nullptr; }
  if (!op->cap_stream) CK(cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking));
  if (!op->body_stream) CK(cudaStreamCreateWithFlags(&op->body_stream, cudaStreamNonBlocking));
  cudaStream_t cs = op->cap_stream, bs = op->body_stream;
  // per-replica residual and right-hand-side norms (one replica unless a stacked batch)
  const int nc = h->ncomp;
  unsigned long long* rbits = h->d_cnorm;
  unsigned long long* fbits = h->d_cnorm + nc;
  amr_status result = AMR_OK;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const long long l0 = g_launches.load();
  do {
    cudaMemsetAsync(op->d_stats, 0, nc * sizeof(DevStats), cs);
    cudaMemsetAsync(rbits, 0, nc * sizeof(unsigned long long), cs);
    if (nc > 1) cudaMemsetAsync(op->d_active, 1, nc * sizeof(int), cs);  // every replica running
    if ((result = composite_op<D>(op, OP_RESID, phi, op->F, op->Res, bc, cs)) != AMR_OK) break;
    if ((result = norm_convert(op, p.precision, rbits, cs)) != AMR_OK) break;
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    cudaGraphConditionalHandle handle;
    if (cudaGraphConditionalHandleCreate(&handle, cg, 0, 0) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    if (nc > 1) launch(k_check_b, 1, 128, 0, cs, handle, 1, nc, rbits, fbits, p.rtol, p.atol, max_steps(p),
                       op->d_stats, op->d_active);
    else launch(k_check, 1, 1, 0, cs, handle, 1, rbits, fbits, p.rtol, p.atol, max_steps(p), op->d_stats);
    if ((result = launch_check()) != AMR_OK) break;
    op->launches_pre = g_launches.load() - l0;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &edata, &ndeps) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, cg, deps, edata, ndeps, &cp) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      result = AMR_ERR_CUDA;
      break;
    }
    const long long l1 = g_launches.load();
    amr_status rb = iteration_body<D>(op, p.precision, p, phi, bc, bs);
    if (rb == AMR_OK) {
      if (nc > 1) launch(k_check_b, 1, 128, 0, bs, handle, 1, nc, rbits, fbits, p.rtol, p.atol, max_steps(p),
                         op->d_stats, op->d_active);
      else launch(k_check, 1, 1, 0, bs, handle, 1, rbits, fbits, p.rtol, p.atol, max_steps(p), op->d_stats);
      rb = launch_check();
    }
    op->launches_body = g_launches.load() - l1;
    cudaGraph_t bout = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(bs, &bout);
    if (rb != AMR_OK) { result = rb; break; }
    if (e1 != cudaSuccess) { set_error(std::string("body capture: ") + cudaGetErrorString(e1)); result = AMR_ERR_CUDA; break; }
    if (cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) {
      result = AMR_ERR_CUDA;
      break;
    }
  } while (false);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  g_launches.store(l0);  // captured launches are counted when the graph runs
  if (result != AMR_OK) {
    if (g) cudaGraphDestroy(g);
    if (std::string(get_error()).empty()) set_error("graph capture failed");
    cudaGetLastError();
    return result;
  }
  if (e2 != cudaSuccess) { set_error(std::string("capture: ") + cudaGetErrorString(e2)); return AMR_ERR_CUDA; }
  op->graph = g;
  CK(cudaGraphInstantiate(&op->exec, g, 0));
  op->g_phi = phi; op->g_bc = bc; op->g_prec = p.precision; op->g_nu1 = p.nu1; op->g_nu2 = p.nu2;
  op->g_maxv = p.max_vcycles; op->g_omega = p.omega; op->g_rtol = p.rtol; op->g_atol = p.atol;
  op->g_fuse = p.fuse_coarse;
  op->g_blk = p.temporal_blocking;
  op->g_cpr = cpr_of(p);
  return AMR_OK;
}

// Captured solve, asynchronous part: set-up, graph launch, epilogue and the stats copy to
// pinned host memory, all on st; solve_graph_finish() reads the stats after a sync.
template <int D>
amr_status solve_graph_launch(amr_operator* op, const amr_solver_params& p, double* phi, const double* f,
                              const double* bc, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  const size_t bytes = (size_t)h->nelems * sizeof(double);
  if (!op->d_stats) {
    const int nc = h->ncomp;
    TRY(dalloc(&op->d_stats, nc));
    if (!op->d_active) TRY(dalloc(&op->d_active, nc));
    CK(cudaMallocHost(&op->h_stats, nc * sizeof(DevStats)));
    CK(cudaMallocHost(&op->h_scal, 8 * sizeof(double)));
    CK(cudaMallocHost(&op->h_cnorm, 2 * nc * sizeof(unsigned long long)));
  }
  if (p.precision == AMR_MIXED) TRY(ensure_scratch<float>(op));
  if (cpr_of(p) > 1) TRY(ensure_inner(op));
  else TRY(ensure_scratch<double>(op));
  CK(cudaMemcpyAsync(op->F, f, bytes, cudaMemcpyDeviceToDevice, st));
  if (op->neumann) {
    TRY(solvability_fix_impl<D>(op, op->F, bc, nullptr, st));
    // keep the removed constant (slot 4 is reused by the final mean-zero)
    CK(cudaMemcpyAsync(h->d_scalar + 6, h->d_scalar + 4, sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  if (p.zero_initial) CK(cudaMemsetAsync(phi, 0, bytes, st));
  TRY(avgdown_all<D>(h, op->F, st));
  // ||f||_inf over the valid cells of every replica
  CK(cudaMemsetAsync(h->d_cnorm + h->ncomp, 0, h->ncomp * sizeof(unsigned long long), st));
  TRY(norm_convert_field(op, op->F, nullptr, h->d_cnorm + h->ncomp, st));
  const bool hit = op->exec && op->g_phi == phi && op->g_bc == bc && op->g_prec == p.precision &&
                   op->g_nu1 == p.nu1 && op->g_nu2 == p.nu2 && op->g_maxv == p.max_vcycles &&
                   op->g_omega == p.omega && op->g_rtol == p.rtol && op->g_atol == p.atol &&
                   op->g_fuse == p.fuse_coarse && op->g_blk == p.temporal_blocking && op->g_cpr == cpr_of(p);
  if (!hit) TRY(build_solve_graph<D>(op, p, phi, bc));
  CK(cudaGraphLaunch(op->exec, st));
  if (op->neumann) TRY(mean_zero_impl<D>(h, phi, nullptr, st));
  else TRY(avgdown_all<D>(h, phi, st));
  CK(cudaMemcpyAsync(op->h_stats, op->d_stats, h->ncomp * sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(op->h_scal, h->d_scalar, 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(op->h_cnorm, h->d_cnorm, 2 * h->ncomp * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  return AMR_OK;
}

// Statistics of replica c of a finished captured solve (c = 0 for a single solve).
amr_status solve_graph_stats(amr_operator* op, int c, amr_solve_stats* stats) {
  const DevStats& ds = op->h_stats[c];
  amr_solve_stats loc{};
  loc.vcycles = ds.iter * op->g_cpr;
  for (int i = 0; i < 64 && i <= ds.iter; ++i) loc.res_history[i] = ds.hist[i];
  loc.final_res = ds.hist[std::min(ds.iter, 63)];
  loc.rhs_norm = __builtin_bit_cast(double, op->h_cnorm[op->h->ncomp + c]);
  loc.removed_mean = op->neumann ? op->h_scal[6] : 0.0;
  if (stats) *stats = loc;
  if (ds.status == 0) return AMR_OK;
  if (ds.status == 2) { set_error("residual is not finite"); return AMR_ERR_NONFINITE; }
  set_error("max_vcycles reached");
  return AMR_ERR_NOT_CONVERGED;
}

amr_status solve_graph_finish(amr_operator* op, amr_solve_stats* stats) {
  TRY(sweep3d_check_flag());
  int most = 0;
  for (int c = 0; c < op->h->ncomp; ++c) most = std::max(most, op->h_stats[c].iter);
  g_launches.fetch_add(op->launches_pre + (long long)most * op->launches_body);
  return solve_graph_stats(op, 0, stats);
}

template <int D>
amr_status solve_graph(amr_operator* op, const amr_solver_params& p, double* phi, const double* f, const double* bc,
                       amr_solve_stats* stats, cudaStream_t st) {
  TRY(solve_graph_launch<D>(op, p, phi, f, bc, st));
  CK(cudaStreamSynchronize(st));
  return solve_graph_finish(op, stats);
}

template <int D>
amr_status apply_transpose_impl(amr_operator* op, const double* y, double* out, cudaStream_t st) {
  TRY(ensure_scratch<double>(op));
  TRY((composite_AT<double, D>(op, y, st)));
  TRY((transpose_residual<double, D>(op, -1, nullptr, out, st)));
  return AMR_OK;
}

template <int D>
amr_status solve_transpose_impl(amr_operator* op, const amr_solver_params& p, double* lam, const double* g,
                                amr_solve_stats* stats, cudaStream_t st) {
  amr_hierarchy* h = op->h;
  const size_t bytes = (size_t)h->nelems * sizeof(double);
  TRY(ensure_scratch<double>(op));
  if (p.precision == AMR_MIXED) TRY(ensure_scratch<float>(op));
  if (cpr_of(p) > 1) TRY(ensure_inner(op));
  amr_solve_stats loc{};
  if (p.zero_initial) CK(cudaMemsetAsync(lam, 0, bytes, st));
  // right-hand side: weight on invalid cells (derived data, the average of their children)
  // is handed to the children by the transposed average-down, coarse to fine
  CK(cudaMemcpyAsync(op->F, g, bytes, cudaMemcpyDeviceToDevice, st));
  for (int l = 0; l + 1 < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.nxfer == 0) continue;
    const int fy = 2 * dl.xfer_max[1];
    const int nby = (fy + BY - 1) / BY;
    dim3 grid((2 * dl.xfer_max[0] + BX - 1) / BX, nby * (D == 3 ? 2 * dl.xfer_max[2] : 1), dl.nxfer);
    launch(k_avgdown_T<double, D>, grid, dim3(BX, BY, 1), 0, st, level_view(h, l + 1, nullptr), level_view(h, l, nullptr),
                                                           dl.xfer, op->F, nby);
    TRY(launch_check());
  }
  g = op->F;
  // pure Neumann: lambda = B^T g with B the bordered solve (solvability correction, solve,
  // mean zero); A^T lambda = F^T g and 1^T lambda = 0 (F^T again at the end)
  if (op->neumann) TRY(neumann_fix_T<D>(h, op->F, &loc.removed_mean, st));
  double gn = 0.0;
  TRY((maxnorm<double, D>(h, g, true, &gn, st)));
  loc.rhs_norm = gn;
  const double tol = std::max(p.rtol * gn, p.atol);
  amr_status result = AMR_ERR_NOT_CONVERGED;
  double res = 0.0;
  int it = 0;
  for (;; ++it) {
    TRY((composite_AT<double, D>(op, lam, st)));
    TRY((transpose_residual<double, D>(op, -1, g, op->Res, st)));
    TRY((maxnorm<double, D>(h, op->Res, true, &res, st)));
    if (it < 64) loc.res_history[it] = res;
    if (!std::isfinite(res)) { result = AMR_ERR_NONFINITE; set_error("residual is not finite"); break; }
    if (res <= tol) { result = AMR_OK; break; }
    if (it >= p.max_vcycles) { set_error("max_vcycles reached"); break; }
    if (p.precision == AMR_MIXED) {
      Scratch<float>& Sf = op->s32;
      for (int l = 0; l < h->L; ++l) TRY((convert<double, float, D>(level_view(h, l, nullptr), op->Res, Sf.rin, st)));
      TRY((vcycle_corr_T<float, D>(op, p, Sf.rin, st)));
      for (int l = 0; l < h->L; ++l) TRY((axpy<float, double, D>(level_view(h, l, nullptr), Sf.X, lam, (double*)nullptr, 1.0, st)));
    } else {
      TRY((vcycle_corr_T<double, D>(op, p, op->Res, st)));
      for (int l = 0; l < h->L; ++l) TRY((axpy<double, double, D>(level_view(h, l, nullptr), op->s64.X, lam, (double*)nullptr, 1.0, st)));
    }
  }
  if (op->neumann) TRY(neumann_fix_T<D>(h, lam, nullptr, st));
  // the adjoint unknowns live on valid cells: zero the invalid ones
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    Geo gg = geo_of(lv);
    launch(k_valid_out<double, D>, gg.grid, gg.block, 0, st, lv, gg.nby, lam, (const double*)nullptr, lam, h->d_valid);
    TRY(launch_check());
  }
  loc.vcycles = it;
  loc.final_res = res;
  if (stats) *stats = loc;
  return result;
}

template <int D>
amr_status vcycle_impl(amr_operator* op, const amr_solver_params& p, double* phi, const double* f, const double* bc,
                       cudaStream_t st) {
  amr_hierarchy* h = op->h;
  TRY(ensure_scratch<double>(op));
  TRY(composite_op<D>(op, OP_RESID, phi, f, op->Res, bc, st));
  TRY(vcycle_corr<double, D>(op, p, op->Res, st));
  for (int l = 0; l < h->L; ++l) TRY(axpy<double, double, D>(level_view(h, l, nullptr), op->s64.X, phi, (double*)nullptr, 1.0, st));
  return AMR_OK;
}

template <int D>
amr_status smooth_impl(amr_operator* op, int level, int nsweeps, double omega, double* x, const double* b,
                       cudaStream_t st) {
  amr_hierarchy* h = op->h;
  TRY(ensure_scratch<double>(op));
  LevelView lv = level_view(h, level, op->bc);
  // zero CF ghosts of x, use Tmp as the ping-pong partner (its CF ghosts zeroed too)
  if (level >= 1) {
    TRY(cfi_fill<double, D>(h, level, x, x, true, st));
    TRY(cfi_fill<double, D>(h, level, op->Tmp, op->Tmp, true, st));
  }
  TRY(smooth_from<double, D>(h, level, lv, b, x, op->Tmp, nsweeps, op->alpha, op->beta, omega, true, st));
  return AMR_OK;
}

// ---------------------------------------------------------------- G, D, projection
template <int D>
amr_status gradient_impl(amr_hierarchy* h, const int* bct, double* phi, double* const* grad, const double* bc,
                         cudaStream_t st) {
  TRY(fill_ghosts_all<D>(h, phi, st));
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, bct);
    Geo g = geo_of(lv);
    launch(k_gradient<double, D>, g.grid, g.block, 0, st, lv, g.nby, phi, grad[0], grad[1], D == 3 ? grad[2] : nullptr, bc);
    TRY(launch_check());
  }
  for (int d = 0; d < D; ++d) TRY(avgdown_all<D>(h, grad[d], st));  // COH-4
  return AMR_OK;
}

template <int D>
amr_status divergence_impl(amr_hierarchy* h, const int* bct, double* const* u, double* out,
                           const double* const* bc, cudaStream_t st) {
  for (int d = 0; d < D; ++d) TRY(fill_ghosts_all<D>(h, u[d], st));
  Ptr3 up{{u[0], u[1], D == 3 ? u[2] : nullptr}};
  Ptr3 bp{{bc ? bc[0] : nullptr, bc ? bc[1] : nullptr, (bc && D == 3) ? bc[2] : nullptr}};
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, bct);
    Geo g = geo_of(lv);
    launch(k_divergence<D>, g.grid, g.block, 0, st, lv, g.nby, up, out, bp);
    TRY(launch_check());
  }
  for (int l = h->L - 2; l >= 0; --l) {
    LevelView c = level_view(h, l, bct), fv = level_view(h, l + 1, bct);
    P3<double> xc{{u[0], u[1], D == 3 ? u[2] : nullptr}};
    P3<double> bcs{{bp.p[0], bp.p[1], bp.p[2]}};
    TRY(reflux<double, D>(h, l, c, fv, xc, xc, bcs, out, 1.0, 1, st));
  }
  TRY(avgdown_all<D>(h, out, st));
  return AMR_OK;
}

template <int D>
amr_status project_impl(amr_operator* ppe, const amr_solver_params& p, const int* vbc, double* const* w,
                        const double* const* wbc, double* const* u, double* phi, amr_solve_stats* stats,
                        cudaStream_t st) {
  amr_hierarchy* h = ppe->h;
  TRY(divergence_impl<D>(h, vbc, w, ppe->Tmp, wbc, st));
  amr_solver_params q = p;
  q.zero_initial = 1;
  amr_status s = solve_impl<D>(ppe, q, phi, ppe->Tmp, nullptr, stats, st);
  if (s != AMR_OK) return s;
  // G^comp phi into u, then u = w - G phi (no average-down of u afterwards)
  TRY(gradient_impl<D>(h, ppe->bc, phi, u, nullptr, st));
  for (int d = 0; d < D; ++d)
    for (int l = 0; l < h->L; ++l) {
      LevelView lv = level_view(h, l, nullptr);
      Geo g = geo_of(lv);
      launch(k_sub<D>, g.grid, g.block, 0, st, lv, g.nby, w[d], u[d], u[d]);
      TRY(launch_check());
    }
  return AMR_OK;
}

// ---------------------------------------------------------------- adjoints of G, D, projection
template <int D>
amr_status ensure_tz(amr_hierarchy* h) {
  if (h->d_tz) return AMR_OK;
  return dalloc(&h->d_tz, (size_t)3 * h->nelems);
}

// Weight on invalid cells of x (outputs of maps that end with an average-down) handed to the
// children, coarse to fine: x <- E^T x in place (invalid entries keep their value).
template <int D>
amr_status avgdown_T_all(amr_hierarchy* h, double* x, cudaStream_t st) {
  for (int l = 0; l + 1 < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.nxfer == 0) continue;
    int nby;
    Geo g = xfer_geo<double, D>(dl, true, nby);
    launch(k_avgdown_T<double, D>, g.grid, dim3(BX, BY, 1), 0, st, level_view(h, l + 1, nullptr), level_view(h, l, nullptr),
                                                             dl.xfer, x, nby);
    TRY(launch_check());
  }
  return AMR_OK;
}

// Adjoints of the ghost fill (COH-1) on a weight field W whose ghost slots hold the weight
// that stencils put on ghost values: copy ghosts -> their sibling cells, CF ghosts -> their
// AMRCFI windows (fine to coarse), then invalid cells -> children (the average-down that
// precedes the ghost fill), then W <- 0 on invalid cells.
template <int D>
amr_status ghost_fill_T(amr_hierarchy* h, double* W, cudaStream_t st) {
  const int nt = 128;
  for (int l = 0; l < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.ncopy == 0) continue;
    launch(k_copy_T<double>, (unsigned)((dl.ncopy + nt - 1) / nt), nt, 0, st, dl.copy, dl.ncopy, W);
    TRY(launch_check());
  }
  for (int l = h->L - 1; l >= 1; --l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.ncfi == 0) continue;
    launch(k_cfi_T<double, D>, (unsigned)((dl.ncfi + nt - 1) / nt), nt, 0, st, 
        dl.cfi, dl.ncfi, dl.cfi_side, h->lev[l - 1].d_patches, h->lev[l].d_patches, h->r, W, W, W, 0.0, 1.0);
    TRY(launch_check());
  }
  TRY(avgdown_T_all<D>(h, W, st));
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    Geo g = geo_of(lv);
    launch(k_valid_out<double, D>, g.grid, g.block, 0, st, lv, g.nby, W, (const double*)nullptr, W, h->d_valid);
    TRY(launch_check());
  }
  return AMR_OK;
}

// out = (G^comp)^T y (sum over components; y's invalid weights handed to children first)
template <int D>
amr_status gradient_T_impl(amr_hierarchy* h, const int* bct, const double* const* y, double* out, cudaStream_t st) {
  TRY(ensure_tz<D>(h));
  const size_t n = (size_t)h->nelems;
  double* Z[3] = {h->d_tz, h->d_tz + n, h->d_tz + 2 * n};
  for (int d = 0; d < D; ++d) {
    CK(cudaMemcpyAsync(Z[d], y[d], n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TRY(avgdown_T_all<D>(h, Z[d], st));
  }
  CK(cudaMemsetAsync(out, 0, n * sizeof(double), st));
  P3c<double> zp{{Z[0], Z[1], Z[2]}};
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, bct);
    Geo g = geo_of(lv);
    launch(k_gradient_T<double, D>, g.grid, g.block, 0, st, lv, g.nby, zp, h->d_valid, out);
    TRY(launch_check());
  }
  return ghost_fill_T<D>(h, out, st);
}

// out[d] = (D^comp)^T y restricted to component d (y's invalid weights handed down first)
template <int D>
amr_status divergence_T_impl(amr_hierarchy* h, const int* bct, const double* y, double* const* out, cudaStream_t st) {
  TRY(ensure_tz<D>(h));
  const size_t n = (size_t)h->nelems;
  double* Z = h->d_tz;
  CK(cudaMemcpyAsync(Z, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(avgdown_T_all<D>(h, Z, st));
  for (int d = 0; d < D; ++d) CK(cudaMemsetAsync(out[d], 0, n * sizeof(double), st));
  Out3<double> W{{out[0], out[1], D == 3 ? out[2] : out[1]}};
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, bct);
    Geo g = geo_of(lv);
    launch(k_divergence_T<double, D>, g.grid, g.block, 0, st, lv, g.nby, Z, h->d_valid, W);
    TRY(launch_check());
  }
  const int nt = 128;
  for (int l = 0; l + 1 < h->L; ++l) {
    const DeviceLists& dl = h->lev[l].dev;
    if (dl.nreflux == 0) continue;
    launch(k_reflux_T<double, D>, (unsigned)((dl.nreflux + nt - 1) / nt), nt, 0, st, 
        level_view(h, l, bct), level_view(h, l + 1, bct), dl.reflux, dl.nreflux, Z, W, 1.0, 1);
    TRY(launch_check());
  }
  for (int d = 0; d < D; ++d) TRY(ghost_fill_T<D>(h, out[d], st));
  return AMR_OK;
}

// out = P^T v for the composite projection u = w - G^comp phi, phi = M D^comp w:
// s = G^T v, lambda = M^T s (adjoint pure-Neumann solve), out_d = v_d - (D^T lambda)_d
// (D^T lambda is 0 on invalid cells, where u_d reads w_d directly).
template <int D>
amr_status project_T_impl(amr_operator* ppe, const amr_solver_params& p, const int* vbc, const double* const* v,
                          double* const* out, double* lam, amr_solve_stats* stats, cudaStream_t st) {
  amr_hierarchy* h = ppe->h;
  TRY(ensure_scratch<double>(ppe));
  TRY(gradient_T_impl<D>(h, ppe->bc, v, ppe->Tmp, st));
  amr_solver_params q = p;
  q.zero_initial = 1;
  amr_status s = solve_transpose_impl<D>(ppe, q, lam, ppe->Tmp, stats, st);
  if (s != AMR_OK) return s;
  TRY(divergence_T_impl<D>(h, vbc, lam, out, st));
  for (int d = 0; d < D; ++d)
    for (int l = 0; l < h->L; ++l) {
      LevelView lv = level_view(h, l, nullptr);
      Geo g = geo_of(lv);
      launch(k_sub<D>, g.grid, g.block, 0, st, lv, g.nby, v[d], out[d], out[d]);
      TRY(launch_check());
    }
  return AMR_OK;
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- work-list batch
// Stopping test of Sec. 7 for every active problem of a work-list batch: records the
// residual norm, retires converged (or failed) problems, and keeps the while-loop of the
// captured batch running while any problem is active.
__global__ void k_check_b(cudaGraphConditionalHandle handle, int use_cond, int n, const unsigned long long* __restrict__ rbits,
                          const unsigned long long* __restrict__ fbits, double rtol, double atol, int maxv,
                          DevStats* __restrict__ s, int* __restrict__ active) {
  pdl_wait();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    if (!active[p]) continue;
    const double r = __longlong_as_double((long long)rbits[p]);
    const double fn = __longlong_as_double((long long)fbits[p]);
    DevStats& st = s[p];
    const int it = st.iter;
    if (it < 64) st.hist[it] = r;
    const double tol = fmax(rtol * fn, atol);
    int cont = 0;
    if (!isfinite(r)) st.status = 2;
    else if (r <= tol) st.status = 0;
    else if (it >= maxv) st.status = 1;
    else {
      cont = 1;
      st.iter = it + 1;
    }
    active[p] = cont;
    if (cont) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(handle, any ? 1u : 0u);
}

// A batch of single-level 2-D problems (mixed precision, temporally blocked legs, square
// coarse pyramids, homogeneous non-Neumann data) solved as one captured graph whose every
// phase is one launch over a descriptor list.
struct BatchGroup {  // one launch: entries [off, off + cnt) of a descriptor array
  int off = 0, cnt = 0, tx = 0, ty = 0, tt = 16;
};
struct BatchPlan {
  std::vector<amr_operator*> ops;
  std::vector<double*> phi;
  std::vector<const double*> f;
  amr_solver_params p{};
  int n = 0, kmax = 0;
  std::vector<BatchGroup> down, up;  // per (m, tile) group, down in increasing m, up in decreasing m
  BatchGroup coarse, resid, flat;
  BDown* d_down = nullptr;
  BUp* d_up = nullptr;
  BCoarse* d_coarse = nullptr;
  BResid* d_resid = nullptr;
  BFlat* d_flat = nullptr;
  int* d_active = nullptr;
  unsigned long long* d_bits = nullptr;  // rbits[n], fbits[n]
  DevStats* d_stats = nullptr;
  DevStats* h_stats = nullptr;  // pinned
  unsigned long long* h_bits = nullptr;  // pinned copy of rbits, fbits
  cudaStream_t cs = nullptr, bs = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches_pre = 0, launches_body = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(d_down); cudaFree(d_up); cudaFree(d_coarse); cudaFree(d_resid); cudaFree(d_flat);
    cudaFree(d_active); cudaFree(d_bits); cudaFree(d_stats);
    if (h_stats) cudaFreeHost(h_stats);
    if (h_bits) cudaFreeHost(h_bits);
    if (cs) cudaStreamDestroy(cs);
    if (bs) cudaStreamDestroy(bs);
    *this = BatchPlan();
  }
};

// levels above the coarse block of op's level-0 pyramid when the batch path applies, else -1
inline int batch_levels(const amr_operator* op, const amr_solver_params& p) {
  const amr_hierarchy* h = op->h;
  if (h->D != 2 || h->L != 1 || h->lev[0].patches.size() != 1 || op->neumann) return -1;
  if (p.precision != AMR_MIXED || !p.temporal_blocking || p.fuse_coarse == 1 || p.nu1 < 1 || p.nu1 > BLK_FX_NU ||
      p.nu2 < 1 || p.nu2 > BLK_FX_NU)
    return -1;
  size_t bytes = 0;
  const int m0 = coarse_block_m0(h, bytes);
  if (m0 < 0) return -1;
  const int M = (int)h->mg.size() - 1;
  if (!square_pyramid(op, m0, M - m0 + 1)) return -1;
  return m0;
}

template <typename D>
amr_status upload(D** dst, const std::vector<D>& v) {
  if (v.empty()) return AMR_OK;
  CK(cudaMalloc(dst, v.size() * sizeof(D)));
  CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(D), cudaMemcpyHostToDevice));
  return AMR_OK;
}

// tile edge of a blocked leg in a batch: many grids at once make the legs throughput-bound,
// where the halo recomputation of a tile (a 36^2 region for 16^2 cells, 52^2 for 32^2) is
// the cost, so the batch takes 32^2 tiles
inline int batch_tile(const int*) { return 32; }

// descriptors of every phase, grouped into launches
amr_status build_batch_lists(BatchPlan& B) {
  const amr_solver_params& p = B.p;
  std::vector<BDown> down;
  std::vector<BUp> up;
  std::vector<BCoarse> coarse;
  std::vector<BResid> resid;
  std::vector<BFlat> flat;
  std::vector<int> K(B.n);
  B.kmax = 0;
  for (int k = 0; k < B.n; ++k) {
    K[k] = batch_levels(B.ops[k], p);
    B.kmax = std::max(B.kmax, K[k]);
  }
  auto group_of = [](std::vector<BatchGroup>& gs, int off, int cnt, int tx, int ty, int tt) {
    if (cnt > 0) gs.push_back(BatchGroup{off, cnt, tx, ty, tt});
  };
  // down legs m = 0 .. kmax-1 and up legs m = kmax-1 .. 0, each split by tile edge
  for (int m = 0; m < B.kmax; ++m)
    for (int tt : {16, 32}) {
      const int off = (int)down.size();
      int tx = 0, ty = 0;
      for (int k = 0; k < B.n; ++k) {
        if (K[k] <= m) continue;
        amr_operator* op = B.ops[k];
        amr_hierarchy* h = op->h;
        if (batch_tile(h->mg[m].n) != tt) continue;
        Scratch<float>& S = op->s32;
        BDown d{};
        d.p = k;
        d.tt = tt;
        d.tiles_x = (h->mg[m].n[0] + tt - 1) / tt;
        d.tiles_y = (h->mg[m].n[1] + tt - 1) / tt;
        d.halo = 2 * p.nu1 + 2;
        d.nu = p.nu1;
        d.lv = mg_view(h, m, op->bc);
        d.gp = h->mg[m].patch;
        d.gcp = h->mg[m + 1].patch;
        d.b = m == 0 ? S.rin : S.mb[m];
        d.xo = m == 0 ? S.T1 : S.mt[m];
        d.bcn = S.mb[m + 1];
        d.alpha = (float)op->alpha;
        d.beta = (float)op->beta;
        d.omega = (float)p.omega;
        d.ood = (float)(p.omega / (op->alpha - 60.0 * op->beta * d.lv.inv12h2));
        tx = std::max(tx, d.tiles_x);
        ty = std::max(ty, d.tiles_y);
        down.push_back(d);
      }
      group_of(B.down, off, (int)down.size() - off, tx, ty, tt);
    }
  for (int m = B.kmax - 1; m >= 0; --m)
    for (int tt : {16, 32}) {
      const int off = (int)up.size();
      int tx = 0, ty = 0;
      for (int k = 0; k < B.n; ++k) {
        if (K[k] <= m) continue;
        amr_operator* op = B.ops[k];
        amr_hierarchy* h = op->h;
        if (batch_tile(h->mg[m].n) != tt) continue;
        Scratch<float>& S = op->s32;
        BUp u{};
        u.p = k;
        u.tt = tt;
        u.tiles_x = (h->mg[m].n[0] + tt - 1) / tt;
        u.tiles_y = (h->mg[m].n[1] + tt - 1) / tt;
        u.halo = 2 * p.nu2;
        u.nu = p.nu2;
        u.lv = mg_view(h, m, op->bc);
        u.cv = mg_view(h, m + 1, op->bc);
        u.gp = h->mg[m].patch;
        u.gcp = h->mg[m + 1].patch;
        u.xc = S.mx[m + 1];
        u.b = m == 0 ? S.rin : S.mb[m];
        u.xi = m == 0 ? S.T1 : S.mt[m];
        u.xo = m == 0 ? S.E : S.mx[m];
        u.alpha = (float)op->alpha;
        u.beta = (float)op->beta;
        u.omega = (float)p.omega;
        u.ood = (float)(p.omega / (op->alpha - 60.0 * op->beta * u.lv.inv12h2));
        tx = std::max(tx, u.tiles_x);
        ty = std::max(ty, u.tiles_y);
        up.push_back(u);
      }
      group_of(B.up, off, (int)up.size() - off, tx, ty, tt);
    }
  int rtx = 0, rty = 0;
  long long nmax = 0;
  for (int k = 0; k < B.n; ++k) {
    amr_operator* op = B.ops[k];
    amr_hierarchy* h = op->h;
    Scratch<float>& S = op->s32;
    const int m0 = K[k];
    BCoarse c{};
    c.p = k;
    c.cb = make_coarse_block(op, p, m0);
    c.n0 = square_pyramid(op, m0, c.cb.ng);
    c.b = m0 == 0 ? S.rin : S.mb[m0];
    c.x = m0 == 0 ? S.E : S.mx[m0];
    c.alpha = (float)op->alpha;
    c.beta = (float)op->beta;
    c.omega = (float)p.omega;
    coarse.push_back(c);
    BResid r{};
    r.p = k;
    r.lv = level_view(h, 0, op->bc);
    r.tiles_x = (r.lv.maxn[0] + BX - 1) / BX;
    r.tiles_y = (r.lv.maxn[1] + BY - 1) / BY;
    r.x = B.phi[k];
    r.f = op->F;
    r.out = op->Res;
    r.alpha = op->alpha;
    r.beta = op->beta;
    rtx = std::max(rtx, r.tiles_x);
    rty = std::max(rty, r.tiles_y);
    resid.push_back(r);
    BFlat fl{};
    fl.p = k;
    fl.n = h->nelems;
    fl.vmask = h->d_valid;
    fl.phi = B.phi[k];
    fl.e = S.E;
    fl.r = op->Res;
    fl.rin = S.rin;
    fl.f = B.f[k];
    fl.F = op->F;
    nmax = std::max(nmax, (long long)h->nelems);
    flat.push_back(fl);
  }
  B.coarse = BatchGroup{0, B.n, 0, 0, 0};
  B.resid = BatchGroup{0, B.n, rtx, rty, 0};
  B.flat = BatchGroup{0, B.n, (int)std::min<long long>((nmax + 255) / 256, 64), 0, 0};
  TRY(upload(&B.d_down, down));
  TRY(upload(&B.d_up, up));
  TRY(upload(&B.d_coarse, coarse));
  TRY(upload(&B.d_resid, resid));
  TRY(upload(&B.d_flat, flat));
  CK(cudaMalloc(&B.d_active, B.n * sizeof(int)));
  CK(cudaMalloc(&B.d_bits, 2 * B.n * sizeof(unsigned long long)));
  CK(cudaMalloc(&B.d_stats, B.n * sizeof(DevStats)));
  CK(cudaMallocHost(&B.h_stats, B.n * sizeof(DevStats)));
  CK(cudaMallocHost(&B.h_bits, 2 * B.n * sizeof(unsigned long long)));
  return AMR_OK;
}

// one V-cycle of every active problem, the update, the new residuals, their norms and the
// stopping test (the body of the captured while-loop)
amr_status batch_body(BatchPlan& B, cudaGraphConditionalHandle handle, cudaStream_t st) {
  const amr_solver_params& p = B.p;
  unsigned long long* rbits = B.d_bits;
  unsigned long long* fbits = B.d_bits + B.n;
  constexpr int RD16 = 16 + 4 * BLK_FX_NU + 4, RD32 = 32 + 4 * BLK_FX_NU + 4;
  constexpr int RU16 = 16 + 4 * BLK_FX_NU, RU32 = 32 + 4 * BLK_FX_NU;
  for (const BatchGroup& g : B.down) {
    const int rm = g.tt == 16 ? RD16 : RD32;
    const size_t smem = (size_t)3 * (rm + 2 * NG) * (rm + 2 * NG) * sizeof(float);
    dim3 grid(g.tx, g.ty, g.cnt);
    if (g.tt == 16) launch(k_mg_down2d_b<RD16, 16>, grid, dim3(32, 8, 1), smem, st, (const BDown*)(B.d_down + g.off), (const int*)B.d_active);
    else launch(k_mg_down2d_b<RD32, 32>, grid, dim3(32, 8, 1), smem, st, (const BDown*)(B.d_down + g.off), (const int*)B.d_active);
    TRY(launch_check());
  }
  launch(k_mg_coarse2d_sq_b, B.coarse.cnt, dim3(32, 32, 1), sizeof(float) * std::max(sq_total<64, 64>(), sq_total<48, 48>()), st,
         (const BCoarse*)B.d_coarse, (const int*)B.d_active);
  TRY(launch_check());
  for (const BatchGroup& g : B.up) {
    const int rm = g.tt == 16 ? RU16 : RU32;
    const size_t smem = (size_t)3 * (rm + 2 * NG) * (rm + 2 * NG) * sizeof(float);
    dim3 grid(g.tx, g.ty, g.cnt);
    if (g.tt == 16) launch(k_mg_up2d_b<RU16, 16>, grid, dim3(32, 8, 1), smem, st, (const BUp*)(B.d_up + g.off), (const int*)B.d_active);
    else launch(k_mg_up2d_b<RU32, 32>, grid, dim3(32, 8, 1), smem, st, (const BUp*)(B.d_up + g.off), (const int*)B.d_active);
    TRY(launch_check());
  }
  launch(k_update_b, dim3(B.flat.tx, B.n, 1), 256, 0, st, (const BFlat*)B.d_flat, (const int*)B.d_active, rbits);
  TRY(launch_check());
  launch(k_resid2d_b<1>, dim3(B.resid.tx, B.resid.ty, B.n), dim3(BX, BY, 1), 0, st, (const BResid*)B.d_resid,
         (const int*)B.d_active);
  TRY(launch_check());
  launch(k_norm_convert_b, dim3(B.flat.tx, B.n, 1), 256, 0, st, (const BFlat*)B.d_flat, (const int*)B.d_active, rbits);
  TRY(launch_check());
  launch(k_check_b, 1, 256, 0, st, handle, 1, B.n, (const unsigned long long*)rbits, (const unsigned long long*)fbits,
         p.rtol, p.atol, p.max_vcycles, B.d_stats, B.d_active);
  return launch_check();
}

amr_status build_batch_graph(BatchPlan& B) {
  const amr_solver_params& p = B.p;
  CK(cudaStreamCreateWithFlags(&B.cs, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&B.bs, cudaStreamNonBlocking));
  unsigned long long* rbits = B.d_bits;
  unsigned long long* fbits = B.d_bits + B.n;
  cudaStream_t cs = B.cs, bs = B.bs;
  amr_status result = AMR_OK;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const long long l0 = g_launches.load();
  do {
    cudaMemsetAsync(B.d_stats, 0, B.n * sizeof(DevStats), cs);
    cudaMemsetAsync(B.d_bits, 0, 2 * B.n * sizeof(unsigned long long), cs);
    cudaMemsetAsync(B.d_active, 1, B.n * sizeof(int), cs);  // nonzero: active
    launch(k_init_b, dim3(B.flat.tx, B.n, 1), 256, 0, cs, (const BFlat*)B.d_flat, p.zero_initial ? 1 : 0, fbits);
    if ((result = launch_check()) != AMR_OK) break;
    launch(k_resid2d_b<1>, dim3(B.resid.tx, B.resid.ty, B.n), dim3(BX, BY, 1), 0, cs, (const BResid*)B.d_resid,
           (const int*)B.d_active);
    if ((result = launch_check()) != AMR_OK) break;
    launch(k_norm_convert_b, dim3(B.flat.tx, B.n, 1), 256, 0, cs, (const BFlat*)B.d_flat, (const int*)B.d_active, rbits);
    if ((result = launch_check()) != AMR_OK) break;
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    cudaGraphConditionalHandle handle;
    if (cudaGraphConditionalHandleCreate(&handle, cg, 0, 0) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    launch(k_check_b, 1, 256, 0, cs, handle, 1, B.n, (const unsigned long long*)rbits, (const unsigned long long*)fbits,
           p.rtol, p.atol, p.max_vcycles, B.d_stats, B.d_active);
    if ((result = launch_check()) != AMR_OK) break;
    B.launches_pre = g_launches.load() - l0;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &edata, &ndeps) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, cg, deps, edata, ndeps, &cp) != cudaSuccess) { result = AMR_ERR_CUDA; break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      result = AMR_ERR_CUDA;
      break;
    }
    const long long l1 = g_launches.load();
    amr_status rb = batch_body(B, handle, bs);
    B.launches_body = g_launches.load() - l1;
    cudaGraph_t bout = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(bs, &bout);
    if (rb != AMR_OK) { result = rb; break; }
    if (e1 != cudaSuccess) { set_error(std::string("batch body capture: ") + cudaGetErrorString(e1)); result = AMR_ERR_CUDA; break; }
    if (cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) {
      result = AMR_ERR_CUDA;
      break;
    }
  } while (false);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  g_launches.store(l0);  // captured launches are counted when the graph runs
  if (result != AMR_OK) {
    if (g) cudaGraphDestroy(g);
    if (std::string(get_error()).empty()) set_error("batch graph capture failed");
    cudaGetLastError();
    return result;
  }
  if (e2 != cudaSuccess) { set_error(std::string("batch capture: ") + cudaGetErrorString(e2)); return AMR_ERR_CUDA; }
  const cudaError_t e3 = cudaGraphInstantiate(&B.exec, g, 0);
  cudaGraphDestroy(g);
  CK(e3);
  return AMR_OK;
}

bool same_params(const amr_solver_params& a, const amr_solver_params& b) {
  return a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.omega == b.omega && a.rtol == b.rtol && a.atol == b.atol &&
         a.max_vcycles == b.max_vcycles && a.precision == b.precision && a.zero_initial == b.zero_initial &&
         a.temporal_blocking == b.temporal_blocking && a.fuse_coarse == b.fuse_coarse;
}

// the batch through the work-list graph; AMR_OK / per-problem status as amr_batch_solve
amr_status batch_worklist(amr_operator* const* ops, int n, const amr_solver_params& q, double* const* phi,
                          const double* const* f, amr_solve_stats* stats, int* status, cudaStream_t st) {
  static std::mutex mu;
  static BatchPlan plan;
  std::lock_guard<std::mutex> lock(mu);
  bool hit = plan.exec && plan.n == n && same_params(plan.p, q);
  for (int k = 0; hit && k < n; ++k) hit = plan.ops[k] == ops[k] && plan.phi[k] == phi[k] && plan.f[k] == f[k];
  if (!hit) {
    plan.release();
    plan.n = n;
    plan.p = q;
    plan.ops.assign(ops, ops + n);
    plan.phi.assign(phi, phi + n);
    plan.f.assign(f, f + n);
    TRY(blk_attrs<float>());
    CK(cudaFuncSetAttribute(k_mg_coarse2d_sq_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    for (int k = 0; k < n; ++k) TRY(ensure_scratch<float>(ops[k]));
    amr_status s = build_batch_lists(plan);
    if (s == AMR_OK) s = build_batch_graph(plan);
    if (s != AMR_OK) { plan.release(); return s; }
  }
  CK(cudaGraphLaunch(plan.exec, st));
  CK(cudaMemcpyAsync(plan.h_stats, plan.d_stats, n * sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(plan.h_bits, plan.d_bits, 2 * n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  amr_status worst = AMR_OK;
  long long iters = 0;
  for (int k = 0; k < n; ++k) {
    const DevStats& ds = plan.h_stats[k];
    iters = std::max<long long>(iters, ds.iter);
    amr_solve_stats loc{};
    loc.vcycles = ds.iter;
    for (int i = 0; i < 64 && i <= ds.iter; ++i) loc.res_history[i] = ds.hist[i];
    loc.final_res = ds.hist[std::min(ds.iter, 63)];
    double fn;
    std::memcpy(&fn, &plan.h_bits[n + k], sizeof(double));
    loc.rhs_norm = fn;
    if (stats) stats[k] = loc;
    const amr_status sk = ds.status == 0 ? AMR_OK : (ds.status == 2 ? AMR_ERR_NONFINITE : AMR_ERR_NOT_CONVERGED);
    if (status) status[k] = sk;
    if (sk != AMR_OK && worst == AMR_OK) {
      worst = sk;
      set_error(sk == AMR_ERR_NONFINITE ? "residual is not finite" : "max_vcycles reached");
    }
  }
  g_launches.fetch_add(plan.launches_pre + iters * plan.launches_body);
  return worst;
}

}  // namespace

// =================================================================== stacked component batches
// A batch of problems that share one 3-D hierarchy geometry and one operator (alpha, beta,
// boundary types; not the pure-Neumann PPE) -- the Helmholtz systems of the velocity
// components -- is solved as one problem on a stacked hierarchy that holds one replica of
// every patch and work list per problem: every phase of the V-cycle and of the refinement
// loop is one launch over all replicas, the stopping test is per replica (a converged
// replica's phi is no longer updated; the loop runs until every replica has converged).
struct StackCtx {
  std::vector<const amr_operator*> key;
  amr_hierarchy* hs = nullptr;
  amr_operator* op = nullptr;
  double* phi = nullptr;
  double* f = nullptr;
};

namespace {

void free_stack(amr_operator* op) {
  if (!op->stack) return;
  StackCtx* c = op->stack;
  cudaFree(c->phi);
  cudaFree(c->f);
  amr_operator_destroy(c->op);
  if (c->hs) {
    free_hierarchy(c->hs);
    delete c->hs;
  }
  delete c;
  op->stack = nullptr;
}

bool same_geometry(const amr_hierarchy* a, const amr_hierarchy* b) {
  if (a->D != b->D || a->r != b->r || a->L != b->L || a->h0 != b->h0 || a->ncomp != 1 || b->ncomp != 1) return false;
  for (int e = 0; e < 3; ++e)
    if (a->n0[e] != b->n0[e]) return false;
  for (int l = 0; l < a->L; ++l) {
    const auto& pa = a->lev[l].patches;
    const auto& pb = b->lev[l].patches;
    if (pa.size() != pb.size()) return false;
    for (size_t k = 0; k < pa.size(); ++k)
      for (int e = 0; e < 3; ++e)
        if (pa[k].n[e] != pb[k].n[e] || pa[k].lo[e] != pb[k].lo[e]) return false;
  }
  return true;
}

// the problems of a batch can be stacked: 3-D, two or more distinct operators on hierarchies
// of one geometry, one operator, homogeneous non-Neumann data
bool stackable(amr_operator* const* ops, int n) {
  if (n < 2 || ops[0]->h->D != 3 || ops[0]->neumann) return false;
  for (int k = 0; k < n; ++k) {
    const amr_operator* a = ops[k];
    if (a->h->ncomp != 1 || a->alpha != ops[0]->alpha || a->beta != ops[0]->beta || !same_geometry(a->h, ops[0]->h))
      return false;
    for (int f = 0; f < 6; ++f)
      if (a->bc[f] != ops[0]->bc[f]) return false;
    for (int j = 0; j < k; ++j)
      if (ops[j] == a) return false;
  }
  return true;
}

amr_status batch_stacked(amr_operator* const* ops, int n, const amr_solver_params& q, double* const* phi,
                         const double* const* f, amr_solve_stats* stats, int* status, cudaStream_t st) {
  amr_operator* lead = ops[0];
  const std::vector<const amr_operator*> key(ops, ops + n);
  if (!lead->stack || lead->stack->key != key) {
    free_stack(lead);
    std::unique_ptr<StackCtx> c(new StackCtx());
    c->key = key;
    std::string err;
    amr_status s1 = stack_hierarchy(lead->h, n, &c->hs, err);
    if (s1 != AMR_OK) {
      set_error(err);
      return s1;
    }
    s1 = amr_operator_create(c->hs, lead->alpha, lead->beta, lead->bc, &c->op);
    if (s1 == AMR_OK) s1 = dalloc(&c->phi, c->hs->nelems);
    // the per-replica running flags of the captured solve (allocated below on the first
    // launch) are what the replica kernels test; allocate them now so views can carry them
    if (s1 == AMR_OK && !c->op->d_active) s1 = dalloc(&c->op->d_active, n);
    if (s1 == AMR_OK) {
      if (cudaMemset(c->op->d_active, 1, n * sizeof(int)) != cudaSuccess) s1 = AMR_ERR_CUDA;
      c->hs->d_active = c->op->d_active;
    }
    if (s1 == AMR_OK) s1 = dalloc(&c->f, c->hs->nelems);
    if (s1 == AMR_OK && (cudaMemset(c->phi, 0, c->hs->nelems * sizeof(double)) != cudaSuccess ||
                         cudaMemset(c->f, 0, c->hs->nelems * sizeof(double)) != cudaSuccess))
      s1 = AMR_ERR_CUDA;
    lead->stack = c.release();
    if (s1 != AMR_OK) {
      free_stack(lead);
      return s1;
    }
  }
  StackCtx* c = lead->stack;
  const long long one = lead->h->nelems, cs = c->hs->cstride;
  for (int k = 0; k < n; ++k) {
    CK(cudaMemcpyAsync(c->f + k * cs, f[k], one * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!q.zero_initial) CK(cudaMemcpyAsync(c->phi + k * cs, phi[k], one * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  TRY(solve_graph_launch<3>(c->op, q, c->phi, c->f, nullptr, st));
  for (int k = 0; k < n; ++k)
    CK(cudaMemcpyAsync(phi[k], c->phi + k * cs, one * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  TRY(sweep3d_check_flag());
  int most = 0;
  for (int k = 0; k < n; ++k) most = std::max(most, c->op->h_stats[k].iter);
  g_launches.fetch_add(c->op->launches_pre + (long long)most * c->op->launches_body);
  amr_status worst = AMR_OK;
  for (int k = 0; k < n; ++k) {
    const amr_status sk = solve_graph_stats(c->op, k, stats ? &stats[k] : nullptr);
    if (status) status[k] = sk;
    if (sk != AMR_OK && worst == AMR_OK) worst = sk;
  }
  return worst;
}
}  // namespace

// =================================================================== allocation-free mean-zero
// Scratch for amr_mean_zero_noalloc: the block partial sums (one double-double per block) and
// three scalars live in this file-scope device array instead of hierarchy-owned memory, so
// the entry point never allocates.  Every GPU that loads the library holds it until exit.
namespace {
constexpr long long NOALLOC_MAX_PARTIALS = 8192;  // largest number of reduction blocks
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_PARTIALS + 8];
std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device
// with that device current (the host-side name is only a stand-in for the device symbol).
// The lookup may initialise the module on that device, which a stream capture does not
// allow, so a first call on a device whose stream is capturing is refused.
amr_status noalloc_scratch(double** out, cudaStream_t st) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("amr_mean_zero_noalloc: device index out of range");
    return AMR_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
      set_error("amr_mean_zero_noalloc: the first call on a device must come before any stream capture (it "
                "looks up the scratch array's device address)");
      return AMR_ERR_INVALID_ARG;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("amr_mean_zero_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return AMR_ERR_CUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return AMR_OK;
}

// The same launches as mean_zero_impl (average-down, k_wsum_gs with the wsum() block count
// per level, k_dd_final, k_mean_from_sums, shift), so the mean and the shifted field are
// bitwise those of amr_mean_zero; only the partials and scalars live in the fixed array.
template <int D>
amr_status mean_zero_noalloc_impl(amr_hierarchy* h, double* x, double* mean_host, cudaStream_t st) {
  // size check before anything is launched
  long long nblocks = 0;
  for (int l = 0; l < h->L; ++l) nblocks += wsum_blocks(level_view(h, l, nullptr));
  if (nblocks > NOALLOC_MAX_PARTIALS) {
    set_error("amr_mean_zero_noalloc: hierarchy needs " + std::to_string(nblocks) +
              " reduction blocks, more than the fixed scratch holds (" + std::to_string(NOALLOC_MAX_PARTIALS) + ")");
    return AMR_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  TRY(noalloc_scratch(&scratch, st));
  double* part = scratch;
  double* sums = scratch + 2 * NOALLOC_MAX_PARTIALS;  // [0] weighted sum, [2] mean
  TRY(avgdown_all<D>(h, x, st));
  long long base = 0;
  for (int l = 0; l < h->L; ++l) {
    LevelView lv = level_view(h, l, nullptr);
    const long long nb = wsum_blocks(lv);
    // every block writes its own partial slot, so no slot needs clearing first
    launch(k_wsum_gs<D>, (unsigned)nb, 256, 0, st, lv, x, h->d_valid, std::pow(lv.h, D), part, base);
    TRY(launch_check());
    base += nb;
  }
  launch(k_dd_final, 1, 256, 0, st, part, base, sums);
  TRY(launch_check());
  launch(k_mean_from_sums, 1, 1, 0, st, sums, nullptr, 0.0, valid_volume(h), sums + 2);
  TRY(launch_check());
  TRY(shift_all<D>(h, x, sums + 2, false, -1.0, st));
  if (mean_host) {
    CK(cudaMemcpyAsync(h->h_scalar + 8, sums + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *mean_host = h->h_scalar[8];
  }
  return AMR_OK;
}

// ---------------------------------------------------------------- interface conditions
// The two rows of I^(4)(k, eta) of Eq. (timeInterp), each entry divided by 6 k^3 (so that
// eta = 0 gives exactly the unit weight on t_{-1}): row 0 the value weights, row 1 those of
// the time derivative, for the data at t_{-i} = t^{l-1} - i k in the order i = 0..3.  The
// printed matrix's columns take the times in increasing order (its entries are the cubic
// Lagrange weights of eta = -2k, -k, 0, k with eta = t* - t_{-1}), so printed column j
// belongs to t_{-(3-j)}.
void cic_weights(double k, double eta, double w[2][4]) {
  const double e = eta, e2 = eta * eta, e3 = e2 * eta, k2 = k * k, k3 = k2 * k, den = 6.0 * k3;
  const double m[2][4] = {{(-e3 + k2 * e) / den, (3.0 * e3 + 3.0 * k * e2 - 6.0 * k2 * e) / den,
                           (-3.0 * e3 - 6.0 * k * e2 + 3.0 * k2 * e + 6.0 * k3) / den,
                           (e3 + 3.0 * k * e2 + 2.0 * k2 * e) / den},
                          {(-3.0 * e2 + k2) / den, (9.0 * e2 + 6.0 * k * e - 6.0 * k2) / den,
                           (-9.0 * e2 - 12.0 * k * e + 3.0 * k2) / den, (3.0 * e2 + 6.0 * k * e + 2.0 * k2) / den}};
  for (int r = 0; r < 2; ++r)
    for (int i = 0; i < 4; ++i) w[r][i] = m[r][3 - i];
}

// The distinct coarse cells of level l's AMRCFI windows and the scratch for their time
// combinations (3-D, ratio 2), made once per level on the first call that needs them.  The
// scratch spans the coarse level's patches (2 doubles per element of that span).
amr_status cic_band(amr_hierarchy* h, int l, cudaStream_t st) {
  LevelHost& L = h->lev[l];
  if (L.dev.cic_y) return AMR_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    set_error("amr_cic_ghosts: the first call for a 3-D level allocates its scratch and must come before any "
              "stream capture");
    return AMR_ERR_INVALID_ARG;
  }
  const LevelHost& C = h->lev[l - 1];
  long long lo = -1, hi = 0;
  for (const PatchDesc& p : C.patches) {
    lo = lo < 0 ? p.off : std::min(lo, p.off);
    hi = std::max(hi, p.off + p.sz * (p.n[2] + 2 * NG));
  }
  std::vector<unsigned char> mark((size_t)(hi - lo), 0);
  for (const CfiEntry& e : L.cfi) {
    if (e.src >= 0) {
      const PatchDesc& cp = C.patches[e.cpatch];
      for (int c2 = 0; c2 < CFI_W; ++c2)
        for (int c1 = 0; c1 < CFI_W; ++c1)
          for (int c0 = 0; c0 < CFI_W; ++c0) mark[(size_t)(e.src + c0 + c1 * cp.sy + c2 * cp.sz - lo)] = 1;
    } else {
      const long long* s = &L.cfi_side[(size_t)(-1 - e.src) * 125];
      for (int q = 0; q < 125; ++q) mark[(size_t)(s[q] - lo)] = 1;
    }
  }
  std::vector<long long> band;
  for (size_t i = 0; i < mark.size(); ++i)
    if (mark[i]) band.push_back(lo + (long long)i);
  long long* d_band = nullptr;
  double* d_y = nullptr;
  if (cudaMalloc(&d_band, sizeof(long long) * std::max<size_t>(band.size(), 1)) != cudaSuccess ||
      cudaMalloc(&d_y, sizeof(double) * 2 * (size_t)(hi - lo)) != cudaSuccess) {
    cudaFree(d_band);
    cudaGetLastError();
    set_error("amr_cic_ghosts: scratch allocation failed");
    return AMR_ERR_OOM;
  }
  CK(cudaMemcpy(d_band, band.data(), sizeof(long long) * band.size(), cudaMemcpyHostToDevice));
  L.dev.cic_band = d_band;
  L.dev.ncic_band = (long long)band.size();
  L.dev.cic_base = lo;
  L.dev.cic_span = hi - lo;
  L.dev.cic_y = d_y;
  return AMR_OK;
}

template <int D>
amr_status cic_ghosts_impl(amr_hierarchy* h, int l, const double* const* xt, double k, double eta, double* v,
                           double* rate, cudaStream_t st) {
  const DeviceLists& dl = h->lev[l].dev;
  if (dl.ncfi == 0) return AMR_OK;
  if (dl.ncfig == 0) {  // ratio 2 groups every CF ghost by its parent
    set_error("amr_cic_ghosts: no parent groups for the CF ghosts");
    return AMR_ERR_INVALID_ARG;
  }
  CicTimes ct{};
  for (int i = 0; i < 4; ++i) ct.x[i] = xt[i];
  cic_weights(k, eta, ct.w);
  const int nt = 128;
  if (D == 3) {
    TRY(cic_band(h, l, st));
    double* y0 = dl.cic_y;
    double* y1 = rate ? dl.cic_y + dl.cic_span : nullptr;
    launch(k_cic_combine, (unsigned)((dl.ncic_band + 255) / 256), 256, 0, st, dl.cic_band, dl.ncic_band,
           dl.cic_base, ct, y0, y1);
    TRY(launch_check());
    launch(k_cic_grp3, (unsigned)((dl.ncfig * CIC_LANES + CIC_GRP_THREADS - 1) / CIC_GRP_THREADS),
           CIC_GRP_THREADS, 0, st, dl.cfig, dl.ncfig, dl.cfi_side, h->lev[l - 1].d_patches, (const double*)y0,
           (const double*)y1, dl.cic_base, v, rate);
  } else {
    launch(k_cic_grp<D>, (unsigned)((dl.ncfig + nt - 1) / nt), nt, 0, st, dl.cfig, dl.ncfig, dl.cfi_side,
           h->lev[l - 1].d_patches, ct, v, rate);
  }
  return launch_check();
}

amr_status cic_faces_impl(amr_hierarchy* h, int l, const double* const* w, const double* phys, double* out,
                          double* delta, cudaStream_t st) {
  const DeviceLists& dl = h->lev[l].dev;
  if (dl.ncic_chunks == 0) return AMR_OK;
  Ptr3 wp{};
  for (int d = 0; d < h->D; ++d) wp.p[d] = w[d];
  launch(k_cic_faces_sum, (unsigned)dl.ncic_chunks, CIC_FACE_THREADS, 0, st, dl.cicf, dl.cic_chunks, wp, out,
         dl.cic_psum);
  TRY(launch_check());
  launch(k_cic_faces_shift, (unsigned)dl.ncic_chunks, CIC_FACE_THREADS, 0, st, dl.cic_chunks, dl.cic_ccstart,
         dl.cic_cstart, dl.cic_psum, phys, out, delta);
  return launch_check();
}

// ---------------------------------------------------------------- data migration
// Device copies of a migration plan, freed when the object goes out of scope.
struct MigrateDev {
  std::vector<void*> ptrs;
  ~MigrateDev() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  amr_status put(const std::vector<T>& v, T** out) {
    *out = nullptr;
    if (v.empty()) return AMR_OK;
    if (cudaMalloc(out, sizeof(T) * v.size()) != cudaSuccess) {
      cudaGetLastError();
      set_error("amr_migrate: device allocation failed");
      return AMR_ERR_OOM;
    }
    ptrs.push_back(*out);
    CK(cudaMemcpy(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return AMR_OK;
  }
};

template <int D>
amr_status migrate_impl(amr_hierarchy* oh, const double* xo, amr_hierarchy* nh, double* xn, cudaStream_t st) {
  std::vector<MigrateLevel> plan;
  std::string err;
  const amr_status ps = migrate_plan(oh, nh, plan, err);
  if (ps != AMR_OK) {
    set_error(err);
    return ps;
  }
  MigrateDev dev;
  unsigned* bad = nullptr;
  TRY(dev.put(std::vector<unsigned>(1, 0u), &bad));
  for (int l = 0; l < nh->L; ++l) {
    const MigrateLevel& M = plan[l];
    MigrateBlock* db = nullptr;
    CfiEntry* dc = nullptr;
    long long* ds = nullptr;
    TRY(dev.put(M.blocks, &db));
    TRY(dev.put(M.cfi, &dc));
    TRY(dev.put(M.side, &ds));
    if (!M.blocks.empty()) {
      long long most = 1;
      for (const MigrateBlock& b : M.blocks) {
        long long c = 1;
        for (int e = 0; e < D; ++e) c *= b.hi[e] - b.lo[e] + 1;
        most = std::max(most, c);
      }
      const unsigned gx = (unsigned)std::min<long long>((most + 255) / 256, 4096);
      launch(k_migrate_copy<D>, dim3(gx, (unsigned)M.blocks.size(), 1), 256, 0, st, (const MigrateBlock*)db,
             (const PatchDesc*)nh->lev[l].d_patches, (const PatchDesc*)oh->lev[l].d_patches, xo, oh->nelems, xn,
             nh->nelems, bad);
      TRY(launch_check());
    }
    if (!M.cfi.empty()) {  // after level l-1 is complete: stream order
      const int nt = 128;
      const long long n = (long long)M.cfi.size();
      launch(k_cfi<double, D>, (unsigned)((n + nt - 1) / nt), nt, 0, st, (const CfiEntry*)dc, n, (const long long*)ds,
             (const PatchDesc*)nh->lev[l - 1].d_patches, nh->r, (const double*)xn, xn, 0);
      TRY(launch_check());
    }
  }
  unsigned nbad = 0;
  CK(cudaMemcpyAsync(&nbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (nbad != 0) {
    set_error("amr_migrate: " + std::to_string(nbad) + " copy offsets outside a field (skipped)");
    return AMR_ERR_INVALID_ARG;
  }
  return AMR_OK;
}
}  // namespace

// =================================================================== C ABI
#define DISPATCH(h, fn, ...) ((h)->D == 2 ? fn<2>(__VA_ARGS__) : fn<3>(__VA_ARGS__))

static amr_status check_op(amr_operator* op) {
  if (op == nullptr || op->h == nullptr) {
    set_error("null operator");
    return AMR_ERR_INVALID_ARG;
  }
  return AMR_OK;
}

static amr_status ensure_device(amr_hierarchy* h) {
  std::string err;
  amr_status s = upload_hierarchy(h, err);
  if (s != AMR_OK) {
    set_error(err);
    return s;
  }
  if (!h->cfi_const_ready) {
    // AMRCFI weights (ratio 2) into this device's constant banks: every entry point that
    // fills CF ghosts (operators, G, D and their transposes) comes through here first
    CK(cudaMemcpyToSymbol(c_cfi, h->cfi_w.data(), h->cfi_w.size() * sizeof(double)));
    std::vector<float> wf(h->cfi_w.begin(), h->cfi_w.end());
    CK(cudaMemcpyToSymbol(c_cfi_f, wf.data(), wf.size() * sizeof(float)));
    h->cfi_const_ready = true;
  }
  return AMR_OK;
}

extern "C" {

const char* amr_last_error(void) { return get_error(); }

long long amr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

amr_status amr_set_tile_rows(int rows) {
  if (rows != 0 && rows != 1 && rows != 2 && rows != 4) { set_error("tile rows must be 0, 1, 2 or 4"); return AMR_ERR_INVALID_ARG; }
  g_tile_force.store(rows, std::memory_order_relaxed);
  return AMR_OK;
}

amr_status amr_set_fx_residual(int on) {
  if (on != 0 && on != 1) { set_error("fixed-point residual switch must be 0 or 1"); return AMR_ERR_INVALID_ARG; }
  g_fx_resid.store(on, std::memory_order_relaxed);
  return AMR_OK;
}

amr_status amr_set_bulk_sweep(int on) {
  if (on < 0 || on > 2) { set_error("bulk-copy sweep switch must be 0, 1 or 2"); return AMR_ERR_INVALID_ARG; }
  g_bulk_sweep.store(on, std::memory_order_relaxed);
  return AMR_OK;
}

amr_status amr_check_kernel_flags(void) { return sweep3d_check_flag(); }

amr_status amr_set_stacked_batches(int on) {
  if (on != 0 && on != 1) { set_error("stacked-batch switch must be 0 or 1"); return AMR_ERR_INVALID_ARG; }
  g_stack_batches.store(on, std::memory_order_relaxed);
  return AMR_OK;
}

amr_status amr_profile_enable(int on) {
  // events are never reused: a cached instrumented graph keeps recording into its own
  if (on) g_prof.recs.clear();
  g_prof.on = on != 0;
  return AMR_OK;
}

amr_status amr_profile_read(int kernel_class, long long* launches, double* total_ms, double* total_bytes) {
  return amr_profile_read_range(kernel_class, 0.0, 1e300, launches, total_ms, total_bytes);
}

amr_status amr_profile_read_range(int kernel_class, double min_cells, double max_cells, long long* launches,
                                  double* total_ms, double* total_bytes) {
  if (kernel_class < 0 || kernel_class >= PC_NCLASS) { set_error("bad kernel class"); return AMR_ERR_INVALID_ARG; }
  long long n = 0;
  double ms = 0.0, by = 0.0;
  for (const ProfRec& r : g_prof.recs) {
    if (r.cls != kernel_class || r.cells < min_cells || r.cells > max_cells) continue;
    CK(cudaEventSynchronize(r.b));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    by += r.bytes;
    ++n;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (total_bytes) *total_bytes = by;
  return AMR_OK;
}

void amr_default_params(amr_solver_params* p) {
  if (!p) return;
  p->nu1 = 4;
  p->nu2 = 4;
  p->omega = 2.0 / 3.0;
  p->rtol = 1e-10;
  p->atol = 0.0;
  p->max_vcycles = 50;
  p->precision = AMR_FP64;
  p->zero_initial = 1;
  p->use_graph = 0;
  p->fuse_coarse = 0;
  p->temporal_blocking = 1;
  p->cycles_per_refinement = 1;
}

amr_status amr_hierarchy_create(const amr_hierarchy_desc* desc, amr_hierarchy** out) {
  if (desc == nullptr || out == nullptr) {
    set_error("null argument");
    return AMR_ERR_INVALID_ARG;
  }
  *out = nullptr;
  amr_hierarchy* h = new (std::nothrow) amr_hierarchy();
  if (!h) {
    set_error("host allocation failed");
    return AMR_ERR_OOM;
  }
  std::string err;
  amr_status st;
  try {
    st = build_hierarchy(desc, h, err);
  } catch (const std::exception& ex) {
    err = ex.what();
    st = AMR_ERR_OOM;
  }
  if (st != AMR_OK) {
    set_error(err);
    free_hierarchy(h);
    delete h;
    return st;
  }
  *out = h;
  return AMR_OK;
}

void amr_hierarchy_destroy(amr_hierarchy* h) {
  if (!h) return;
  free_hierarchy(h);
  delete h;
}

amr_status amr_field_layout(const amr_hierarchy* h, int* npatches, long long* nelems, amr_patch_info* patches) {
  if (!h) { set_error("null hierarchy"); return AMR_ERR_INVALID_ARG; }
  if (npatches) *npatches = h->npatch;
  if (nelems) *nelems = h->nelems;
  if (patches) std::memcpy(patches, h->pinfo.data(), h->pinfo.size() * sizeof(amr_patch_info));
  return AMR_OK;
}

amr_status amr_bc_layout(const amr_hierarchy* h, long long* offsets) {
  if (!h || !offsets) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  std::memcpy(offsets, h->bc_off.data(), h->bc_off.size() * sizeof(long long));
  return AMR_OK;
}

amr_status amr_get_index_maps(const amr_hierarchy* h, amr_index_maps* o) {
  if (!h || !o) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  o->ncells_interior = (long long)h->im_valid.size();
  o->ncells_padded = (long long)h->im_code.size();
  o->valid = h->im_valid.data();
  o->component = h->im_component.data();
  o->ghost_code = h->im_code.data();
  o->ghost_src = h->im_src.data();
  o->ghost_aux = h->im_aux.data();
  o->ncfi = (long long)h->im_cfi_cell.size();
  o->cfi_cell = h->im_cfi_cell.data();
  o->cfi_start = h->im_cfi_start.data();
  o->cfi_pos = h->im_cfi_pos.data();
  o->cfi_sub = h->im_cfi_sub.data();
  o->nreflux = (long long)h->im_reflux_faces.size();
  o->reflux_cell = h->im_reflux_cell.data();
  o->reflux_faces = h->im_reflux_faces.data();
  return AMR_OK;
}

amr_status amr_operator_create(amr_hierarchy* h, double alpha, double beta, const int* bc_types, amr_operator** out) {
  if (!h || !bc_types || !out) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  *out = nullptr;
  if (h->r != 2) { set_error("solver calls need refinement ratio 2"); return AMR_ERR_INVALID_ARG; }
  for (int f = 0; f < 2 * h->D; ++f)
    if (bc_types[f] != AMR_BC_DIRICHLET && bc_types[f] != AMR_BC_NEUMANN) { set_error("bad bc type"); return AMR_ERR_INVALID_ARG; }
  if (!std::isfinite(alpha) || !std::isfinite(beta) || beta == 0.0) { set_error("bad alpha/beta"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  std::unique_ptr<amr_operator> op(new amr_operator());
  op->h = h;
  op->alpha = alpha;
  op->beta = beta;
  bool alln = true;
  for (int f = 0; f < 6; ++f) op->bc[f] = f < 2 * h->D ? bc_types[f] : 0;
  for (int f = 0; f < 2 * h->D; ++f) alln = alln && bc_types[f] == AMR_BC_NEUMANN;
  op->neumann = alln && alpha == 0.0;
  // dense bottom inverse on the coarsest level-0 multigrid grid
  const MgGrid& g = h->mg.back();
  const int n = g.n[0] * g.n[1] * g.n[2];
  const int ld = op->neumann ? n + 1 : n;
  std::vector<double> A((size_t)ld * ld, 0.0);
  std::vector<double> e(n, 0.0), y;
  for (int j = 0; j < n; ++j) {
    e.assign(n, 0.0);
    e[j] = 1.0;
    host_apply(h->D, g.n, g.h, alpha, beta, op->bc, e, y);
    for (int i = 0; i < n; ++i) A[(size_t)i * ld + j] = y[i];
  }
  if (op->neumann) {
    for (int i = 0; i < n; ++i) { A[(size_t)i * ld + n] = 1.0; A[(size_t)n * ld + i] = 1.0; }
  }
  if (!invert(A, ld)) { set_error("singular bottom operator"); return AMR_ERR_INVALID_ARG; }
  op->nbot = n;
  op->ldb = ld;
  TRY(dalloc(&op->d_binv, A.size()));
  CK(cudaMemcpy(op->d_binv, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice));
  {
    std::vector<double> At(A.size());
    for (int i = 0; i < ld; ++i)
      for (int j2 = 0; j2 < ld; ++j2) At[(size_t)i * ld + j2] = A[(size_t)j2 * ld + i];
    TRY(dalloc(&op->d_binvT, At.size()));
    CK(cudaMemcpy(op->d_binvT, At.data(), At.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  // multigrid transfer blocks (one per replica of a stacked component batch)
  for (size_t m = 0; m + 1 < h->mg.size(); ++m) {
    std::vector<XferBlock> bs(h->ncomp);
    for (int c = 0; c < h->ncomp; ++c) {
      XferBlock& b = bs[c];
      b = XferBlock{};
      b.fpatch = c;
      b.cpatch = c;
      for (int q = 0; q < 3; ++q) { b.clo[q] = 0; b.chi[q] = h->mg[m + 1].n[q] - 1; }
    }
    XferBlock* d = nullptr;
    TRY(dalloc(&d, bs.size()));
    CK(cudaMemcpy(d, bs.data(), bs.size() * sizeof(XferBlock), cudaMemcpyHostToDevice));
    op->d_mgx.push_back(d);
  }
  const size_t ne = (size_t)h->nelems;
  TRY(dalloc(&op->F, ne));
  TRY(dalloc(&op->Res, ne));
  TRY(dalloc(&op->Tmp, ne));
  CK(cudaMemset(op->F, 0, ne * sizeof(double)));
  CK(cudaMemset(op->Res, 0, ne * sizeof(double)));
  CK(cudaMemset(op->Tmp, 0, ne * sizeof(double)));
  *out = op.release();
  return AMR_OK;
}

void amr_operator_destroy(amr_operator* op) {
  if (!op) return;
  free_scratch(op->s64);
  free_scratch(op->s32);
  cudaFree(op->d_binv);
  cudaFree(op->d_binvT);
  cudaFree(op->F);
  cudaFree(op->Res);
  cudaFree(op->Tmp);
  for (auto p : op->d_mgx) cudaFree(p);
  cudaFree(op->hphi);
  cudaFree(op->inner_x);
  cudaFree(op->inner_r);
  cudaFree(op->hf);
  cudaFree(op->hbc);
  if (op->exec) cudaGraphExecDestroy(op->exec);
  if (op->graph) cudaGraphDestroy(op->graph);
  if (op->cap_stream) cudaStreamDestroy(op->cap_stream);
  if (op->body_stream) cudaStreamDestroy(op->body_stream);
  cudaFree(op->d_stats);
  cudaFree(op->d_active);
  if (op->h_stats) cudaFreeHost(op->h_stats);
  if (op->h_scal) cudaFreeHost(op->h_scal);
  if (op->h_cnorm) cudaFreeHost(op->h_cnorm);
  free_stack(op);
  delete op;
}

amr_status amr_fill_ghosts(amr_operator* op, double* phi, const double* bc, void* stream) {
  TRY(check_op(op));
  if (!phi) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  (void)bc;  // physical ghosts are evaluated on the fly by the operators; see below
  amr_hierarchy* h = op->h;
  TRY(DISPATCH(h, fill_ghosts_all, h, phi, S(stream)));
  return AMR_OK;
}

static amr_status check_cic_level(const amr_hierarchy* h, int level) {
  if (!h) { set_error("null hierarchy"); return AMR_ERR_INVALID_ARG; }
  if (h->ncomp != 1) { set_error("interface conditions need an unstacked hierarchy"); return AMR_ERR_INVALID_ARG; }
  if (h->r != 2) { set_error("interface conditions need refinement ratio 2"); return AMR_ERR_INVALID_ARG; }
  if (level < 1 || level >= h->L) {
    set_error("interface conditions: level " + std::to_string(level) + " is not a refined level (1.." +
              std::to_string(h->L - 1) + ")");
    return AMR_ERR_INVALID_ARG;
  }
  return AMR_OK;
}

amr_status amr_cic_ghosts(amr_hierarchy* h, int level, const double* const* coarse, double k, double eta,
                          double* value, double* rate, void* stream) {
  TRY(check_cic_level(h, level));
  if (!coarse || !value) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  for (int i = 0; i < 4; ++i)
    if (!coarse[i]) { set_error("amr_cic_ghosts: null coarse time level"); return AMR_ERR_INVALID_ARG; }
  if (!(k > 0.0) || !std::isfinite(k) || !std::isfinite(eta)) {
    set_error("amr_cic_ghosts: needs a finite time step k > 0 and a finite eta");
    return AMR_ERR_INVALID_ARG;
  }
  TRY(ensure_device(h));
  return DISPATCH(h, cic_ghosts_impl, h, level, coarse, k, eta, value, rate, S(stream));
}

amr_status amr_cic_faces(const amr_hierarchy* h, int level, int* nfaces, int* ncomponents, int* cell, int* face,
                         int* component) {
  TRY(check_cic_level(h, level));
  const LevelHost& L = h->lev[level];
  const int nf = (int)L.cicf.size();
  if (nfaces) *nfaces = nf;
  if (ncomponents) *ncomponents = L.cic_cstart.empty() ? 0 : (int)L.cic_cstart.size() - 1;
  if (cell) std::memcpy(cell, L.cic_cell.data(), L.cic_cell.size() * sizeof(int));
  if (face)
    for (int i = 0; i < nf; ++i) face[i] = 2 * L.cicf[i].dir + (L.cicf[i].side > 0 ? 1 : 0);
  if (component) std::memcpy(component, L.cic_comp.data(), L.cic_comp.size() * sizeof(int));
  return AMR_OK;
}

amr_status amr_migrate(amr_hierarchy* old_h, const double* old_x, amr_hierarchy* new_h, double* new_x,
                       void* stream) {
  if (!old_h || !old_x || !new_h || !new_x) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  if (old_x == new_x) { set_error("amr_migrate: the old and new fields must be different buffers"); return AMR_ERR_INVALID_ARG; }
  if (new_h->r != 2) { set_error("amr_migrate: needs refinement ratio 2"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(old_h));
  TRY(ensure_device(new_h));
  return DISPATCH(new_h, migrate_impl, old_h, old_x, new_h, new_x, S(stream));
}

amr_status amr_migrate_plan(const amr_hierarchy* old_h, const amr_hierarchy* new_h, int level, int* nblocks,
                            int* blocks, long long* ncells, int* cells, int* starts, long long* dst, long long* src,
                            long long* nside, long long* side) {
  if (!old_h || !new_h) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  if (level < 0 || level >= new_h->L) { set_error("amr_migrate_plan: level out of range"); return AMR_ERR_INVALID_ARG; }
  std::vector<MigrateLevel> plan;
  std::string err;
  const amr_status ps = migrate_plan(old_h, new_h, plan, err);
  if (ps != AMR_OK) {
    set_error(err);
    return ps;
  }
  const MigrateLevel& M = plan[level];
  const int D = new_h->D;
  if (nblocks) *nblocks = (int)M.blocks.size();
  if (blocks)
    for (size_t i = 0; i < M.blocks.size(); ++i) {
      int* q = blocks + i * (2 + 2 * D);
      q[0] = M.blocks[i].npatch;
      q[1] = M.blocks[i].opatch;
      for (int e = 0; e < D; ++e) {
        q[2 + e] = M.blocks[i].lo[e];
        q[2 + D + e] = M.blocks[i].hi[e];
      }
    }
  if (ncells) *ncells = (long long)M.cfi.size();
  if (cells) std::memcpy(cells, M.cells.data(), M.cells.size() * sizeof(int));
  if (starts) std::memcpy(starts, M.starts.data(), M.starts.size() * sizeof(int));
  if (dst)
    for (size_t i = 0; i < M.cfi.size(); ++i) dst[i] = M.cfi[i].dst;
  if (src)
    for (size_t i = 0; i < M.cfi.size(); ++i) src[i] = M.cfi[i].src;
  if (nside) *nside = (long long)M.side.size();
  if (side) std::memcpy(side, M.side.data(), M.side.size() * sizeof(long long));
  return AMR_OK;
}

amr_status amr_cic_component_box(const amr_hierarchy* h, int level, int component, int* lo, int* hi,
                                 int* interface_faces) {
  TRY(check_cic_level(h, level));
  const LevelHost& L = h->lev[level];
  if (component < 0 || component >= (int)L.cic_comp_box.size()) {
    set_error("amr_cic_component_box: component out of range");
    return AMR_ERR_INVALID_ARG;
  }
  const int b = L.cic_comp_box[component];
  if (b < 0) {
    set_error("amr_cic_component_box: component " + std::to_string(component) + " of level " + std::to_string(level) +
              " has several boxes (its level problem is not a box problem)");
    return AMR_ERR_INVALID_ARG;
  }
  const Box& B = L.boxes[b];
  for (int d = 0; d < h->D; ++d) {
    if (lo) lo[d] = B.lo[d];
    if (hi) hi[d] = B.hi[d];
    if (interface_faces) {
      interface_faces[2 * d] = B.lo[d] > 0 ? 1 : 0;
      interface_faces[2 * d + 1] = B.hi[d] < L.ndom[d] - 1 ? 1 : 0;
    }
  }
  return AMR_OK;
}

amr_status amr_cic_interface_bc(amr_hierarchy* h, int level, int component, const double* x, double* bc,
                                void* stream) {
  TRY(amr_cic_component_box(h, level, component, nullptr, nullptr, nullptr));
  if (!x || !bc) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  const LevelHost& L = h->lev[level];
  const int b = L.cic_cstart[component], e = L.cic_cstart[component + 1];
  if (e == b) return AMR_OK;
  const int nt = 256;
  launch(k_cic_face_bc, (unsigned)((e - b + nt - 1) / nt), nt, 0, S(stream), L.dev.cicf, L.dev.cic_slot, b, e, x, bc);
  return launch_check();
}

amr_status amr_cic_face_averages(amr_hierarchy* h, int level, const double* const* w, const double* phys,
                                 double* faces, double* delta, void* stream) {
  TRY(check_cic_level(h, level));
  if (!w || (!faces && !h->lev[level].cicf.empty())) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  for (int d = 0; d < h->D; ++d)
    if (!w[d]) { set_error("amr_cic_face_averages: null velocity component"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  return cic_faces_impl(h, level, w, phys, faces, delta, S(stream));
}

amr_status amr_apply(amr_operator* op, double* phi, double* out, const double* bc, void* stream) {
  TRY(check_op(op));
  if (!phi || !out) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(DISPATCH(op->h, composite_op, op, OP_APPLY, phi, (const double*)nullptr, out, bc, S(stream)));
  return AMR_OK;
}

amr_status amr_residual(amr_operator* op, double* phi, const double* f, double* res, const double* bc, double* norm,
                        void* stream) {
  TRY(check_op(op));
  if (!phi || !f || !res) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(DISPATCH(op->h, composite_op, op, OP_RESID, phi, f, res, bc, S(stream)));
  if (norm) {
    amr_hierarchy* h = op->h;
    if (h->D == 2) TRY((maxnorm<double, 2>(h, res, true, norm, S(stream))));
    else TRY((maxnorm<double, 3>(h, res, true, norm, S(stream))));
  }
  return AMR_OK;
}

amr_status amr_smooth(amr_operator* op, int level, int nsweeps, double omega, double* x, const double* b, void* stream) {
  TRY(check_op(op));
  if (level < 0 || level >= op->h->L || nsweeps < 0 || !x || !b) { set_error("bad argument"); return AMR_ERR_INVALID_ARG; }
  TRY(DISPATCH(op->h, smooth_impl, op, level, nsweeps, omega, x, b, S(stream)));
  return AMR_OK;
}

static amr_status check_params(const amr_solver_params* p) {
  if (!p || p->nu1 < 0 || p->nu2 < 0 || p->max_vcycles < 0 || !(p->omega > 0.0) ||
      (p->precision != AMR_FP64 && p->precision != AMR_MIXED) || p->fuse_coarse < 0 || p->fuse_coarse > 2 ||
      p->cycles_per_refinement < 1 || p->cycles_per_refinement > 4) {
    set_error("bad solver parameters");
    return AMR_ERR_INVALID_ARG;
  }
  return AMR_OK;
}

amr_status amr_vcycle(amr_operator* op, const amr_solver_params* p, double* phi, const double* f, const double* bc,
                      void* stream) {
  TRY(check_op(op));
  TRY(check_params(p));
  if (!phi || !f) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(DISPATCH(op->h, vcycle_impl, op, *p, phi, f, bc, S(stream)));
  return AMR_OK;
}

amr_status amr_solve(amr_operator* op, const amr_solver_params* p, double* phi, const double* f, const double* bc,
                     amr_solve_stats* stats, void* stream) {
  TRY(check_op(op));
  TRY(check_params(p));
  if (!phi || !f) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  return DISPATCH(op->h, solve_impl, op, *p, phi, f, bc, stats, S(stream));
}

amr_status amr_solve_host(amr_operator* op, const amr_solver_params* p, double* phi_host, const double* f_host,
                          const double* bc_host, amr_solve_stats* stats, void* stream) {
  TRY(check_op(op));
  TRY(check_params(p));
  if (!phi_host || !f_host) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  amr_hierarchy* h = op->h;
  const size_t bytes = (size_t)h->nelems * sizeof(double);
  cudaStream_t st = S(stream);
  const size_t nbc = (size_t)h->bc_off.back();
  if (!op->hphi) TRY(dalloc(&op->hphi, h->nelems));
  if (!op->hf) TRY(dalloc(&op->hf, h->nelems));
  if (bc_host && !op->hbc) TRY(dalloc(&op->hbc, nbc));
  CK(cudaMemcpyAsync(op->hf, f_host, bytes, cudaMemcpyHostToDevice, st));
  if (!p->zero_initial) CK(cudaMemcpyAsync(op->hphi, phi_host, bytes, cudaMemcpyHostToDevice, st));
  if (bc_host) CK(cudaMemcpyAsync(op->hbc, bc_host, nbc * sizeof(double), cudaMemcpyHostToDevice, st));
  amr_status s = DISPATCH(h, solve_impl, op, *p, op->hphi, op->hf, bc_host ? op->hbc : nullptr, stats, st);
  if (s == AMR_OK || s == AMR_ERR_NOT_CONVERGED) {
    CK(cudaMemcpyAsync(phi_host, op->hphi, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return s;
}

// The batch solve; with f_host / phi_host (amr_batch_solve_host, device staging phi / f) the
// concurrent per-problem path copies each problem's data on its own stream around its solve.
// The caller of the host form makes f_host, phi_host null for the other paths.
amr_status batch_solve_impl(amr_operator* const* ops, int n, const amr_solver_params* p, double* const* phi,
                            const double* const* f, amr_solve_stats* stats, int* status, void* stream,
                            const double* const* f_host = nullptr, double* const* phi_host = nullptr);

amr_status amr_batch_solve(amr_operator* const* ops, int n, const amr_solver_params* p, double* const* phi,
                           const double* const* f, amr_solve_stats* stats, int* status, void* stream) {
  return batch_solve_impl(ops, n, p, phi, f, stats, status, stream);
}

amr_status batch_solve_impl(amr_operator* const* ops, int n, const amr_solver_params* p, double* const* phi,
                            const double* const* f, amr_solve_stats* stats, int* status, void* stream,
                            const double* const* f_host, double* const* phi_host) {
  if (!ops || n < 0 || !phi || !f) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  TRY(check_params(p));
  for (int k = 0; k < n; ++k) {
    TRY(check_op(ops[k]));
    if (!phi[k] || !f[k]) { set_error("null field in batch"); return AMR_ERR_INVALID_ARG; }
  }
  static std::mutex mu;
  static std::vector<cudaStream_t> pool;
  static std::vector<cudaEvent_t> ev;
  constexpr int NSTREAM = 16;
  if (pool.empty()) {
    pool.resize(NSTREAM);
    ev.resize(NSTREAM + 1);
    for (int i = 0; i < NSTREAM; ++i) CK(cudaStreamCreateWithFlags(&pool[i], cudaStreamNonBlocking));
    for (auto& e : ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t st = S(stream);
  amr_solver_params q = *p;
  q.use_graph = 1;
  // single-level 2-D problems with blocked legs: one launch per phase over a work list; one
  // 3-D geometry and operator for every problem: one stacked solve
  bool worklist = n > 0;
  for (int k = 0; k < n && worklist; ++k) worklist = batch_levels(ops[k], q) >= 0;
  const bool stacked = !worklist && g_stack_batches.load(std::memory_order_relaxed) && stackable(ops, n);
  if (worklist || stacked) {
    // host buffers: all copies in, the batch, all copies out, on the caller's stream
    for (int k = 0; k < n && f_host != nullptr; ++k) {
      const size_t bytes = (size_t)ops[k]->h->nelems * sizeof(double);
      CK(cudaMemcpyAsync(const_cast<double*>(f[k]), f_host[k], bytes, cudaMemcpyHostToDevice, st));
      if (!q.zero_initial) CK(cudaMemcpyAsync(phi[k], phi_host[k], bytes, cudaMemcpyHostToDevice, st));
    }
    const amr_status s = worklist ? batch_worklist(ops, n, q, phi, f, stats, status, st)
                                  : batch_stacked(ops, n, q, phi, f, stats, status, st);
    if (phi_host == nullptr || (s != AMR_OK && s != AMR_ERR_NOT_CONVERGED)) return s;
    for (int k = 0; k < n; ++k)
      CK(cudaMemcpyAsync(phi_host[k], phi[k], (size_t)ops[k]->h->nelems * sizeof(double), cudaMemcpyDeviceToHost,
                         st));
    CK(cudaStreamSynchronize(st));
    return s;
  }
  std::lock_guard<std::mutex> lock(mu);
  // problems that share a hierarchy share its reduction scratch: same stream, in order
  std::vector<const amr_hierarchy*> hs;
  std::vector<int> sid(n);
  for (int k = 0; k < n; ++k) {
    auto it = std::find(hs.begin(), hs.end(), ops[k]->h);
    const int hidx = (int)(it - hs.begin());
    if (it == hs.end()) hs.push_back(ops[k]->h);
    sid[k] = hidx % NSTREAM;
  }
  CK(cudaEventRecord(ev[NSTREAM], st));
  for (int i = 0; i < NSTREAM; ++i) CK(cudaStreamWaitEvent(pool[i], ev[NSTREAM], 0));
  for (int k = 0; k < n; ++k) {
    amr_operator* op = ops[k];
    cudaStream_t sk = pool[sid[k]];
    const size_t bytes = (size_t)op->h->nelems * sizeof(double);
    // host buffers (amr_batch_solve_host): each problem's copies sit on its own stream, so the
    // copies of one problem overlap the solves of the others
    if (f_host != nullptr) {
      CK(cudaMemcpyAsync(const_cast<double*>(f[k]), f_host[k], bytes, cudaMemcpyHostToDevice, sk));
      if (!q.zero_initial) CK(cudaMemcpyAsync(phi[k], phi_host[k], bytes, cudaMemcpyHostToDevice, sk));
    }
    TRY(DISPATCH(op->h, solve_graph_launch, op, q, phi[k], f[k], nullptr, sk));
    if (phi_host != nullptr) CK(cudaMemcpyAsync(phi_host[k], phi[k], bytes, cudaMemcpyDeviceToHost, sk));
  }
  for (int i = 0; i < NSTREAM; ++i) {
    CK(cudaEventRecord(ev[i], pool[i]));
    CK(cudaStreamWaitEvent(st, ev[i], 0));
  }
  CK(cudaStreamSynchronize(st));
  amr_status worst = AMR_OK;
  for (int k = 0; k < n; ++k) {
    amr_status sk = solve_graph_finish(ops[k], stats ? &stats[k] : nullptr);
    if (status) status[k] = sk;
    if (sk != AMR_OK && worst == AMR_OK) worst = sk;
  }
  return worst;
}

amr_status amr_batch_solve_host(amr_operator* const* ops, int n, const amr_solver_params* p, double* const* phi_host,
                                const double* const* f_host, amr_solve_stats* stats, int* status, void* stream) {
  if (!ops || n < 0 || !phi_host || !f_host) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  TRY(check_params(p));
  for (int k = 0; k < n; ++k) {
    TRY(check_op(ops[k]));
    if (!phi_host[k] || !f_host[k]) { set_error("null field in batch"); return AMR_ERR_INVALID_ARG; }
    for (int j = 0; j < k; ++j)
      if (ops[j] == ops[k]) { set_error("an operator appears twice in a host-buffer batch"); return AMR_ERR_INVALID_ARG; }
  }
  std::vector<double*> dphi(n);
  std::vector<const double*> df(n);
  for (int k = 0; k < n; ++k) {
    amr_operator* op = ops[k];
    if (!op->hphi) TRY(dalloc(&op->hphi, op->h->nelems));
    if (!op->hf) TRY(dalloc(&op->hf, op->h->nelems));
    dphi[k] = op->hphi;
    df[k] = op->hf;
  }
  // the copies are issued by the batch itself (per problem and stream where it runs the
  // problems concurrently), and the call returns once every phi is back on the host
  const amr_status s = batch_solve_impl(ops, n, p, dphi.data(), df.data(), stats, status, stream, f_host, phi_host);
  CK(cudaStreamSynchronize(S(stream)));
  return s;
}

amr_status amr_solvability_fix(amr_operator* op, double* f, const double* bc, double* m, void* stream) {
  TRY(check_op(op));
  if (!f) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(DISPATCH(op->h, solvability_fix_impl, op, f, bc, m, S(stream)));
  return AMR_OK;
}

amr_status amr_mean_zero(amr_hierarchy* h, double* phi, double* mean, void* stream) {
  if (!h || !phi) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  TRY(DISPATCH(h, mean_zero_impl, h, phi, mean, S(stream)));
  return AMR_OK;
}

amr_status amr_mean_zero_noalloc(amr_hierarchy* h, double* phi, double* mean, void* stream) {
  if (!h || !phi) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  if (!h->on_device) {
    set_error("amr_mean_zero_noalloc: the hierarchy has no device copy yet (create an operator or call another "
              "device entry point once beforehand)");
    return AMR_ERR_INVALID_ARG;
  }
  return DISPATCH(h, mean_zero_noalloc_impl, h, phi, mean, S(stream));
}

amr_status amr_gradient(amr_hierarchy* h, const int* bc_types, double* phi, double* const* grad, const double* bc,
                        void* stream) {
  if (!h || !bc_types || !phi || !grad) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  TRY(DISPATCH(h, gradient_impl, h, bc_types, phi, grad, bc, S(stream)));
  return AMR_OK;
}

amr_status amr_divergence(amr_hierarchy* h, const int* bc_types, double* const* u, double* out, const double* const* bc,
                          void* stream) {
  if (!h || !bc_types || !u || !out) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  TRY(DISPATCH(h, divergence_impl, h, bc_types, u, out, bc, S(stream)));
  return AMR_OK;
}

amr_status amr_project(amr_operator* ppe, const amr_solver_params* p, const int* vel_bc_types, double* const* w,
                       const double* const* w_bc, double* const* u, double* phi, amr_solve_stats* stats, void* stream) {
  TRY(check_op(ppe));
  TRY(check_params(p));
  if (!ppe->neumann) { set_error("projection needs the pure-Neumann PPE operator"); return AMR_ERR_INVALID_ARG; }
  if (!vel_bc_types || !w || !u || !phi) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  return DISPATCH(ppe->h, project_impl, ppe, *p, vel_bc_types, w, w_bc, u, phi, stats, S(stream));
}

amr_status amr_apply_transpose(amr_operator* op, const double* y, double* out, void* stream) {
  TRY(check_op(op));
  if (!y || !out) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(DISPATCH(op->h, apply_transpose_impl, op, y, out, S(stream)));
  return AMR_OK;
}

amr_status amr_solve_transpose(amr_operator* op, const amr_solver_params* p, double* lambda, const double* g,
                               amr_solve_stats* stats, void* stream) {
  TRY(check_op(op));
  TRY(check_params(p));
  if (!lambda || !g) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  return DISPATCH(op->h, solve_transpose_impl, op, *p, lambda, g, stats, S(stream));
}

amr_status amr_gradient_transpose(amr_hierarchy* h, const int* bc_types, const double* const* y, double* out,
                                  void* stream) {
  if (!h || !bc_types || !y || !out) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  for (int d = 0; d < h->D; ++d)
    if (!y[d]) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  return DISPATCH(h, gradient_T_impl, h, bc_types, y, out, S(stream));
}

amr_status amr_divergence_transpose(amr_hierarchy* h, const int* bc_types, const double* y, double* const* out,
                                    void* stream) {
  if (!h || !bc_types || !y || !out) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  for (int d = 0; d < h->D; ++d)
    if (!out[d]) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  TRY(ensure_device(h));
  return DISPATCH(h, divergence_T_impl, h, bc_types, y, out, S(stream));
}

amr_status amr_project_transpose(amr_operator* ppe, const amr_solver_params* p, const int* vel_bc_types,
                                 const double* const* v, double* const* out, double* lambda, amr_solve_stats* stats,
                                 void* stream) {
  TRY(check_op(ppe));
  TRY(check_params(p));
  if (!ppe->neumann) { set_error("projection needs the pure-Neumann PPE operator"); return AMR_ERR_INVALID_ARG; }
  if (!vel_bc_types || !v || !out || !lambda) { set_error("null argument"); return AMR_ERR_INVALID_ARG; }
  for (int d = 0; d < ppe->h->D; ++d)
    if (!v[d] || !out[d]) { set_error("null field"); return AMR_ERR_INVALID_ARG; }
  return DISPATCH(ppe->h, project_T_impl, ppe, *p, vel_bc_types, v, out, lambda, stats, S(stream));
}

}  // extern "C"
