// Host runtime and C ABI of the kappa-cycle multigrid (declared in include/kcycle.h).
//
// The handle owns the level hierarchy (per level: current estimate, right-hand side and a
// temporary, Section 3.1), the per-level Galerkin stencils computed on the device, and a cache of
// CUDA graphs. A cycle is Algorithm 3 unrolled on the host into kernel launches for the fine
// levels -- pass A before the recursive calls, pass B after -- while every call at or below the
// coarse threshold is one launch of the single-CTA coarse kernel, which walks the rest of the
// recursion on the device. The launch sequence of a cycle is captured once into a graph and
// replayed; stand-alone solves and MGCG put one cycle (or one PCG iteration) in the body of a
// WHILE conditional node whose last kernel evaluates the stopping test on the device, so a whole
// solve is a single graph launch.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <list>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/kcycle.h"
#include "kernels.cuh"
#include "lines.cuh"
#include "stream_f32.cuh"
#include "tma_f32.cuh"
#include "deep.cuh"

using namespace kc;

namespace {

thread_local char g_err[256] = "";

#define KC_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      snprintf(g_err, sizeof(g_err), "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
               __FILE__, __LINE__);                                                         \
      return e_ == cudaErrorMemoryAllocation ? MG_ERR_NOMEM : MG_ERR_CUDA;                  \
    }                                                                                       \
  } while (0)

#define KC_TRY(expr)          \
  do {                        \
    int s_ = (expr);          \
    if (s_ < 0) return s_;    \
  } while (0)

constexpr int NT_SMALL = 256;
constexpr int NT_TINY = 128;
constexpr int NT_BIG = 512;
constexpr int NT_COARSE = 256;     // coarse kernel, FP64 (bound by the SM's FP64 pipe)
constexpr int NT_COARSE32 = 512;   // coarse kernel, FP32 (latency bound: more threads per phase)
template <typename T>
constexpr int nt_coarse() { return std::is_same<T, double>::value ? NT_COARSE : NT_COARSE32; }
constexpr int NT_VEC = 256;
constexpr int NT_DEEP = 256;  // persistent deep calls: threads per CTA (one or two CTAs per SM)
constexpr int MAX_NU = 8;
constexpr int VEC_BLOCKS = 148 * 8;
constexpr int MAX_COARSE_N = 63;
constexpr size_t SMEM_CAP = 220 * 1024;  // dynamic shared memory per CTA (227 KB less static use)
// Output rows per tile of the tensor-copy FP32 passes (pass A from zero, pass A from v, pass B): the
// window (tile plus halo rows, double-buffered) sized so that three, two and two CTAs of 8 warps
// share an SM, whose copies and barriers then overlap each other's arithmetic.
constexpr int TMA_TY_A0 = 32, TMA_TY_A = 24, TMA_TY_B = 32;
constexpr int TMA_TY_S = 8, TMA_SMALL_MAX = 511;  // tile height at the small sides (255, 511)
constexpr int TMA_MIN_N = 255;                     // smallest side for the tensor-copy passes
constexpr int MAP_S = 49;       // unknowns of the side-7 level
constexpr int MAP_CLASSES = 3;  // at most two levels below it: counters 1, 2, >= 3

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Level {
  int n = 0, ld = 0;      // rows (the side, except under semi-coarsening) and pitch
  int nx = 0;             // columns: n, or the finest side at every level under semi-coarsening
  double* v = nullptr;    // current estimate (level 0: the caller's array)
  double* tmp = nullptr;  // relaxed v between pass A and pass B
  double* f = nullptr;    // right-hand side (level 0: the caller's array)
  // FP32 hierarchy of the mixed-precision cycle, allocated on first use; level 0 holds the
  // FP32 correction d (v32) and the rounded FP64 residual (f32)
  float* v32 = nullptr;
  float* tmp32 = nullptr;
  float* f32 = nullptr;
};

enum GraphKind { G_CYCLE = 1, G_SOLVE = 2, G_PCG = 3, G_CYCLE32 = 4, G_MIXED = 5 };

struct GraphEntry {
  int kind = 0, kappa = 0, flag = 0;
  const void* p0 = nullptr;
  const void* p1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
};

// Per-call pointer binding of level 0 (caller memory) over the handle's own levels.
template <typename T>
struct BindingT {
  T* v0;
  const T* f0;
  int ld0;
};
using Binding = BindingT<double>;

}  // namespace

struct mg_ctx {
  int n = 0, k = 0, levels = 0, nu1 = 2, nu2 = 2;
  double eps = 0, theta = 0, omega = 0.8;
  int coarse_n = 31;  // largest side handled by the coarse kernel (FP64 cycles); its two child calls
                      // of each call at 63^2 run as the condensed 961 x 961 product over ~120 CTAs
                      // (measured at 4095^2 against 15: kappa=4 solve 1,860 -> 1,716 ms, every
                      // kappa and the zebra and MGCG settings faster or equal)
  int lc = 0;         // first level handled by the coarse kernel (FP64 cycles)
  int lc32 = 0;       // same for the FP32 cycles of the mixed path
  int fused = 1;         // calls one (1) or two (2) levels above the coarse kernel as one cluster launch
                         // (MG_OPT_FUSED_CALL)
  int tma32 = 1;         // FP32 large-level passes fed by tensor copies (MG_OPT_TMA_PASSES)
  int sms = 148;         // multiprocessors of the device (grid of the persistent passes)
  int coarse_n32 = 31;  // FP32 threshold: one SM does FP32 at 64x the FP64 rate, so the single-CTA
                        // kernel takes more levels (31 measured best at 4095^2 for kappa 3 and 4)
  Level lv[MAXL];
  double* coef = nullptr;
  float* coef32 = nullptr;
  double* stencils = nullptr;   // MAXL*9
  double* dstencil = nullptr;   // 18: d/dtheta, d/deps of the fine stencil
  double* cinv = nullptr;
  float* cinv32 = nullptr;
  double* work = nullptr;
  double* partial = nullptr;
  double* partial2 = nullptr;
  size_t npartial = 0;
  double* scal = nullptr;
  int* ints = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  bool have32 = false;  // FP32 hierarchy allocated
  int ld32_0 = 0;       // pitch of the FP32 level-0 arrays (multiple of 32 floats)
  int rediscretized = 0;  // coarse operators: 0 Galerkin, 1 the Section 4 stencil on each coarse grid
  int stop_rule = 0;      // 0: ||f - A v|| / ||f|| <= tol; 1: ||v_k|| / ||v_0|| <= tol (f = 0 protocol)
  int smoother = 0;       // 0 damped Jacobi, 1 alternating zebra line Gauss-Seidel, 2 zebra along x only
  int semi = 0;           // 1: semi-coarsening along y (every level keeps the n columns)
  int precond = 0;        // MGCG preconditioner: 0 the kappa-cycle B, 1 B + B^T - B^T A B
  double bx = 0.0, by = 0.0;  // upwind convection b . grad u (Section 5's non-symmetric problem)
  bool nonsym = false;        // bx or by nonzero: general-stencil kernels, FP64 damped Jacobi only
  // condensed coarse calls: the affine maps of a call at the side-7 level, per counter class, for
  // the FP64 and FP32 coarse kernels (valid while the flags are set)
  double* cmap = nullptr;
  float* cmap32 = nullptr;
  bool maps_ok = false, maps32_ok = false;
  // condensed child calls at the coarse-kernel level (children_kernel): per class c = 1..pm_cls the
  // map P_c (pm_side^2 rows of pitch pm_ld), FP64 and FP32 cycles; valid while pm_ok / pm32_ok
  int condense = 1;  // MG_OPT_CONDENSED_CHILDREN
  int stall_tile = -1;  // MG_OPT_TEST_STALL_COPY
  int stall_cta = -1;   // MG_OPT_TEST_STALL_BARRIER
  int deep_n = 127;     // MG_OPT_DEEP_CALLS: calls at sides <= deep_n as one persistent launch (0: off);
                        // measured at 4095^2: mixed solves 2-6% faster, FP64 solves unchanged
  bool batched = false;  // an instance of a batch: its graph branch runs beside the others'
  double* pm = nullptr;
  float* pm32 = nullptr;
  int pm_cls = 0, pm_ld = 0, pm_side = 0, pm32_cls = 0, pm32_ld = 0, pm32_side = 0;
  bool pm_ok = false, pm32_ok = false;
  double* ltab = nullptr;  // line-solve tables (Thomas factors and chunk products) per level/direction
  float* ltab32 = nullptr;
  double* linv = nullptr;  // dense line inverses of the levels with side <= LINV_MAX
  double *pr = nullptr, *pp = nullptr, *pq = nullptr, *pz = nullptr, *pzold = nullptr;  // PCG vectors
  double *pw = nullptr, *pz2 = nullptr;  // symmetrised preconditioner: r - A B r and B^T (r - A B r)
  double *hv = nullptr, *hf = nullptr;  // device copies for mg_solve_host
  cudaStream_t own = nullptr;
  cudaStream_t ext = nullptr;
  bool has_ext = false;
  std::list<GraphEntry> graphs;  // stable addresses; trimmed only at the start of a public call
  int last_launches = 0;
  int launch_count = 0;  // counter while emitting
  bool ok = false;
  // per-launch timing (mg_profile_cycle): an event pair around each launch while `prof` is set
  bool prof = false;
  bool prof_graph = false;  // profiling inside a stream capture (external event records)
  std::vector<cudaEvent_t> pev;
  std::vector<int> pkind, plevel;

  cudaStream_t stream() const { return has_ext ? ext : own; }
};

namespace {

// ------------------------------------------------------------------------------------------
// Tile configurations per level size
// ------------------------------------------------------------------------------------------
template <int BX, int BY, int NT>
struct TileCfg {
  static constexpr int bx = BX, by = BY, nt = NT;
};
// 64 x 48 (94 KB of FP64 shared memory, two CTAs per SM) for the passes that also sum squared
// residuals (the level-0 pass A of a stand-alone solve: its first sweep in the residual form);
// 64 x 32 (66 KB, three CTAs per SM) for the others. Measured at 4095^2: the summing pass A 1.18 ms
// with 64 x 48 against 1.24 ms with 64 x 32; pass B 947 -> 937 us and the 2047^2 passes
// 261 -> 253 us (A) and 255 -> 241 us (B) with 64 x 32.
using Tile64 = TileCfg<64, 48, NT_BIG>;
using Tile64N = TileCfg<64, 32, NT_BIG>;
using Tile32 = TileCfg<32, 32, NT_SMALL>;
using Tile16 = TileCfg<16, 16, NT_TINY>;
using Tile8 = TileCfg<8, 8, NT_TINY>;

// FP64 level passes are bound by the FP64 pipe of each SM, so a launch must spread over all SMs:
// take the largest tile that still gives about two waves of CTAs at edge 64 and one wave at
// edges 32 and 16 (measured: the smaller tiles' halo recomputation costs more than the imbalance
// of a single wave at 511^2 and 255^2).
int tile_edge(int n) {
  for (int b : {64, 32, 16}) {
    const int g = (n + b - 1) / b;
    if (g * g >= (b == 64 ? 2 : 1) * 148) return b;
  }
  return 8;
}
// rows of the tile of a pass at side n: `sums` for the passes that write residual sums
int tile_rows(int n, bool sums = true) { return tile_edge(n) == 64 ? (sums ? 48 : 32) : tile_edge(n); }

// FP64 levels below level 0 that one tile per SM covers: the smallest even tile edge whose tiles
// number at most the SMs, where that edge is an instantiated one (on 148 SMs: 511^2 in 12 x 12
// tiles of 44^2, 255^2 in 12 x 12 tiles of 22^2), instead of tile_edge's 256 tiles, of which most
// SMs would run two on their FP64 pipe. 0: none. Not for the instances of a batch: their passes
// share the SMs with the other instances' (the 44^2 pass B's 512 threads take an SM's whole
// register file; measured, the FP64 batch 10.52 -> 10.75 s with them).
using Tile44 = TileCfg<44, 44, NT_BIG>;
using Tile22 = TileCfg<22, 22, NT_SMALL>;
int wide_edge(int n, int sms) {
  for (int b = 2; b <= 64; b += 2) {
    const int g = (n + b - 1) / b;
    if (g * g <= sms) return (b == 44 || b == 22) ? b : 0;
  }
  return 0;
}

// ns: the general (non-symmetric) stencil variant, FP64 only.
template <typename Cfg, typename T>
int launch_pass_a(const PassAArgs<T>& a, cudaStream_t s, bool ns = false) {
  dim3 grid((a.n + Cfg::bx - 1) / Cfg::bx, (a.n + Cfg::by - 1) / Cfg::by);
  const size_t sm = pass_a_smem<T, Cfg::bx, Cfg::by>(a.nu);
  if constexpr (std::is_same<T, double>::value) {
    if (ns) {
      pass_a_kernel<T, Cfg::bx, Cfg::by, Cfg::nt, true><<<grid, Cfg::nt, sm, s>>>(a);
      KC_CUDA(cudaGetLastError());
      return MG_OK;
    }
  }
  if (ns) return MG_ERR_ARG;
  pass_a_kernel<T, Cfg::bx, Cfg::by, Cfg::nt><<<grid, Cfg::nt, sm, s>>>(a);
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}
template <typename Cfg, typename T>
int launch_pass_b(const PassBArgs<T>& a, cudaStream_t s, bool ns = false) {
  dim3 grid((a.n + Cfg::bx - 1) / Cfg::bx, (a.n + Cfg::by - 1) / Cfg::by);
  const size_t sm = pass_b_smem<T, Cfg::bx, Cfg::by>(a.nu, a.partial != nullptr);
  if constexpr (std::is_same<T, double>::value) {
    if (ns) {
      pass_b_kernel<T, Cfg::bx, Cfg::by, Cfg::nt, true><<<grid, Cfg::nt, sm, s>>>(a);
      KC_CUDA(cudaGetLastError());
      return MG_OK;
    }
  }
  if (ns) return MG_ERR_ARG;
  pass_b_kernel<T, Cfg::bx, Cfg::by, Cfg::nt><<<grid, Cfg::nt, sm, s>>>(a);
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

template <typename Cfg, typename T>
int set_smem_attrs() {
  KC_CUDA(cudaFuncSetAttribute(pass_a_kernel<T, Cfg::bx, Cfg::by, Cfg::nt>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)pass_a_smem<T, Cfg::bx, Cfg::by>(MAX_NU)));
  KC_CUDA(cudaFuncSetAttribute(pass_b_kernel<T, Cfg::bx, Cfg::by, Cfg::nt>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)pass_b_smem<T, Cfg::bx, Cfg::by>(MAX_NU, true)));
  if constexpr (std::is_same<T, double>::value) {
    KC_CUDA(cudaFuncSetAttribute(pass_a_kernel<T, Cfg::bx, Cfg::by, Cfg::nt, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pass_a_smem<T, Cfg::bx, Cfg::by>(MAX_NU)));
    KC_CUDA(cudaFuncSetAttribute(pass_b_kernel<T, Cfg::bx, Cfg::by, Cfg::nt, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pass_b_smem<T, Cfg::bx, Cfg::by>(MAX_NU, true)));
  }
  return MG_OK;
}

constexpr int LINE_R = 4;  // lines per CTA of the zebra line kernels

template <typename T, int MC>
int set_line_attrs() {
  KC_CUDA(cudaFuncSetAttribute(line_relax_kernel<T, 0, LINE_R, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)line_smem<T, LINE_R, MC>()));
  KC_CUDA(cudaFuncSetAttribute(line_relax_kernel<T, 1, LINE_R, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)line_smem<T, LINE_R, MC>()));
  return MG_OK;
}

// The largest dynamic shared memory a coarse walk asks for: its levels (up to side MAX_COARSE_N),
// plus the condensed-call maps where they fit under SMEM_CAP.
template <typename T>
size_t coarse_smem_max() {
  return std::min(SMEM_CAP, coarse_smem<T>(MAX_COARSE_N, 6) + coarse_map_smem<T>(MAP_CLASSES));
}

template <typename T>
int set_all_smem_attrs() {
  KC_TRY((set_smem_attrs<Tile64, T>()));
  KC_TRY((set_smem_attrs<Tile64N, T>()));
  KC_TRY((set_smem_attrs<Tile32, T>()));
  KC_TRY((set_smem_attrs<Tile16, T>()));
  KC_TRY((set_smem_attrs<Tile8, T>()));
  if constexpr (std::is_same<T, double>::value) {
    KC_TRY((set_smem_attrs<Tile44, T>()));
    KC_TRY((set_smem_attrs<Tile22, T>()));
  }
  KC_CUDA(cudaFuncSetAttribute(coarse_kernel<T, nt_coarse<T>(), false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)coarse_smem_max<T>()));
  KC_CUDA(cudaFuncSetAttribute(coarse_kernel<T, nt_coarse<T>(), true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)coarse_smem_max<T>()));
  if constexpr (std::is_same<T, double>::value) {
    KC_CUDA(cudaFuncSetAttribute(coarse_kernel<T, nt_coarse<T>(), false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coarse_smem_max<T>()));
  }
  if constexpr (std::is_same<T, float>::value) {
    for (auto k : {pass_a_tile32<0>, pass_a_tile32<1>, pass_a_tile32<2>})
      KC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile32_smem_a()));
    for (auto k : {pass_b_tile32<0>, pass_b_tile32<1>, pass_b_tile32<2>})
      KC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile32_smem_b()));
    KC_CUDA(cudaFuncSetAttribute(pass_a_tma32<true, TMA_TY_A0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tm_smem_a(TMA_TY_A0, 2, true) + 1024)));
    KC_CUDA(cudaFuncSetAttribute(pass_a_tma32<false, TMA_TY_A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tm_smem_a(TMA_TY_A, 2, false) + 1024)));
    KC_CUDA(cudaFuncSetAttribute(pass_b_tma32<TMA_TY_B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tm_smem_b(TMA_TY_B, 2) + 1024)));
    KC_CUDA(cudaFuncSetAttribute(pass_a_tma32<true, TMA_TY_S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tm_smem_a(TMA_TY_S, 2, true) + 1024)));
    KC_CUDA(cudaFuncSetAttribute(pass_a_tma32<false, TMA_TY_S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tm_smem_a(TMA_TY_S, 2, false) + 1024)));
    KC_CUDA(cudaFuncSetAttribute(pass_b_tma32<TMA_TY_S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tm_smem_b(TMA_TY_S, 2) + 1024)));
  }
  KC_TRY((set_line_attrs<T, 1>()));
  KC_TRY((set_line_attrs<T, 2>()));
  KC_TRY((set_line_attrs<T, 4>()));
  KC_TRY((set_line_attrs<T, 8>()));
  KC_TRY((set_line_attrs<T, 16>()));
  return MG_OK;
}

size_t pass_grid_blocks(int n) {
  return (size_t)((n + tile_edge(n) - 1) / tile_edge(n)) * (size_t)((n + tile_rows(n) - 1) / tile_rows(n));
}

size_t apply_grid_blocks(int n) {
  return size_t((n + 31) / 32) * size_t((n + NT_VEC / 32 - 1) / (NT_VEC / 32));
}

// ------------------------------------------------------------------------------------------
// Cycle emission (Algorithm 3 unrolled over the fine levels)
// ------------------------------------------------------------------------------------------
// Level arrays of one precision: the FP64 hierarchy or the FP32 one of the mixed cycle.
template <typename T>
struct Arr;
template <>
struct Arr<double> {
  static double* v(mg_ctx* h, int l) { return h->lv[l].v; }
  static double* tmp(mg_ctx* h, int l) { return h->lv[l].tmp; }
  static double* f(mg_ctx* h, int l) { return h->lv[l].f; }
  static const double* coef(mg_ctx* h) { return h->coef; }
  static const double* ltab(mg_ctx* h) { return h->ltab; }
  static double* cmap(mg_ctx* h) { return h->cmap; }
  static bool maps_ok(mg_ctx* h) { return h->maps_ok; }
  static int ld(mg_ctx* h, int l) { return h->lv[l].ld; }
  static const double* pmap(const mg_ctx* h, int c, int* ld) {
    if (!h->pm_ok || !h->condense) return nullptr;
    *ld = h->pm_ld;
    return h->pm + (size_t)(std::min(c, h->pm_cls) - 1) * h->pm_side * h->pm_side * h->pm_ld;
  }
};
template <>
struct Arr<float> {
  static float* v(mg_ctx* h, int l) { return h->lv[l].v32; }
  static float* tmp(mg_ctx* h, int l) { return h->lv[l].tmp32; }
  static float* f(mg_ctx* h, int l) { return h->lv[l].f32; }
  static const float* coef(mg_ctx* h) { return h->coef32; }
  static const float* ltab(mg_ctx* h) { return h->ltab32; }
  static float* cmap(mg_ctx* h) { return h->cmap32; }
  static bool maps_ok(mg_ctx* h) { return h->maps32_ok; }
  static int ld(mg_ctx* h, int l) { return l == 0 ? h->ld32_0 : h->lv[l].ld; }
  static const float* pmap(const mg_ctx* h, int c, int* ld) {
    if (!h->pm32_ok || !h->condense) return nullptr;
    *ld = h->pm32_ld;
    return h->pm32 + (size_t)(std::min(c, h->pm32_cls) - 1) * h->pm32_side * h->pm32_side * h->pm32_ld;
  }
};

template <typename T>
int lc_of(const mg_ctx* h) { return std::is_same<T, double>::value ? h->lc : h->lc32; }

template <typename T>
T* lv_v(mg_ctx* h, const BindingT<T>& b, int l) { return l == 0 ? b.v0 : Arr<T>::v(h, l); }
template <typename T>
const T* lv_f(mg_ctx* h, const BindingT<T>& b, int l) { return l == 0 ? b.f0 : Arr<T>::f(h, l); }
template <typename T>
int lv_ld(mg_ctx* h, const BindingT<T>& b, int l) { return l == 0 ? b.ld0 : Arr<T>::ld(h, l); }

enum { K_PASS_A = 0, K_PASS_B = 1, K_COARSE = 2, K_APPLY = 3, K_LINES_X = 4, K_LINES_Y = 5, K_CALL = 6, K_DEEP = 7 };
// (under semi-coarsening K_PASS_A is the y restriction and K_PASS_B the y prolongation)

// Inside a stream capture an event record must be an external one to become a graph node whose
// time cudaEventElapsedTime reads.
void prof_record(mg_ctx* h, cudaEvent_t e, cudaStream_t s) {
  if (h->prof_graph) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}
void prof_begin(mg_ctx* h, int kind, int level, cudaStream_t s) {
  if (!h->prof) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  prof_record(h, e, s);
  h->pev.push_back(e);
  h->pkind.push_back(kind);
  h->plevel.push_back(level);
}
void prof_end(mg_ctx* h, cudaStream_t s) {
  if (!h->prof) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  prof_record(h, e, s);
  h->pev.push_back(e);
}

// FP32 fast passes (register pipeline, shared-memory tiles): large levels, nu <= 2, 16-byte
// aligned rows with a pitch multiple of 4.
constexpr int F32_FAST_MIN = 1023;  // smallest side for the FP32 pipelines or shared-memory tiles
bool fast32_ok(int n, int nu, const void* p, int ld) {
  return n >= F32_FAST_MIN && nu <= 2 && (p == nullptr || ((uintptr_t)p & 15) == 0) && (ld & 3) == 0;
}
int stream_rows(int n) { return n >= 4095 ? 64 : (n >= 2047 ? 32 : 16); }

// FP32 passes at the fast-eligible levels: the shared-memory tile passes (112 x 16 outputs per
// CTA) for pass A, and for pass B below side 4095; the register pipeline for pass B from 4095 up.
// Measured in the FP32 cycle of the 4095^2 mixed solve: at 4095^2 pass A 83 -> 76 us with tiles
// (against the register pipeline it replaced), pass B 107 us with the pipeline against 114 with
// tiles (whose loads are not overlapped within a CTA); at 2047^2 pass A 39 -> 28 us and pass B 40
// -> 32 us (the pipelines' grid gives 9 warps per SM there); at 1023^2 17 -> 13 and 18 -> 14 us
// against the generic tiles.
bool f32_tile_pass_b(int n) { return n < 4095; }

int launch_pass_a_tile32(const PassAArgs<float>& a, cudaStream_t s) {
  dim3 grid((a.n + T32_TX - 1) / T32_TX, (a.n + T32_TY - 1) / T32_TY);
  const size_t sm = tile32_smem_a();
  switch (a.nu) {
    case 0: pass_a_tile32<0><<<grid, T32_NT, sm, s>>>(a); break;
    case 1: pass_a_tile32<1><<<grid, T32_NT, sm, s>>>(a); break;
    default: pass_a_tile32<2><<<grid, T32_NT, sm, s>>>(a); break;
  }
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}
int launch_pass_b_tile32(const PassBArgs<float>& a, cudaStream_t s) {
  dim3 grid((a.n + T32_TX - 1) / T32_TX, (a.n + T32_TY - 1) / T32_TY);
  const size_t sm = tile32_smem_b();
  switch (a.nu) {
    case 0: pass_b_tile32<0><<<grid, T32_NT, sm, s>>>(a); break;
    case 1: pass_b_tile32<1><<<grid, T32_NT, sm, s>>>(a); break;
    default: pass_b_tile32<2><<<grid, T32_NT, sm, s>>>(a); break;
  }
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

int launch_pass_b_fast32(const PassBArgs<float>& a, cudaStream_t s) {
  if (f32_tile_pass_b(a.n)) return launch_pass_b_tile32(a, s);
  const int strips = (a.n + SF_COLS - 1) / SF_COLS, R = stream_rows(a.n);
  dim3 grid((strips + SF_WARPS - 1) / SF_WARPS, (a.n + R - 1) / R);
  switch (a.nu) {
    case 0: pass_b_stream_f32<0, false><<<grid, 32 * SF_WARPS, 0, s>>>(a, R); break;
    case 1: pass_b_stream_f32<1, false><<<grid, 32 * SF_WARPS, 0, s>>>(a, R); break;
    default: pass_b_stream_f32<2, false><<<grid, 32 * SF_WARPS, 0, s>>>(a, R); break;
  }
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

// ------------------------------------------------------------------------------------------
// FP32 passes fed by tensor copies (tma_f32.cuh): tensor maps and launches
// ------------------------------------------------------------------------------------------
// The driver's tensor-map encoder, looked up once through the runtime (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// A 2-D map of an n_cols x n_rows FP32 array (row pitch ld floats) read in box_x x box_y boxes;
// points outside the extents read as zero.
int make_map_f32(CUtensorMap* m, const float* base, int n_cols, int n_rows, int ld, int box_x, int box_y) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return MG_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)n_cols, (cuuint64_t)n_rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(g_err, sizeof(g_err), "cuTensorMapEncodeTiled failed (%d) for a %d x %d array, pitch %d", (int)r, n_cols,
             n_rows, ld);
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

// Kinds of tensor-copy pass; TMA_SMALL + kind: the same pass with tiles of TMA_TY_S rows, used at the
// sides up to TMA_SMALL_MAX, where tall tiles would leave most SMs without a tile.
enum TmaKind { TMA_A_ZERO = 0, TMA_A = 1, TMA_B = 2, TMA_SMALL = 3 };
int tma_kind(int base, int n) { return n <= TMA_SMALL_MAX ? TMA_SMALL + base : base; }
int tma_ty(int kind) {
  if (kind >= TMA_SMALL) return TMA_TY_S;
  return kind == TMA_A ? TMA_TY_A : (kind == TMA_B ? TMA_TY_B : TMA_TY_A0);
}
size_t tma_smem(int kind) {
  const int base = kind % TMA_SMALL;
  return (base == TMA_B ? tm_smem_b(tma_ty(kind), 2) : tm_smem_a(tma_ty(kind), 2, base == TMA_A_ZERO)) + 1024;
}

// CTAs of a tensor-copy pass: every resident slot of the device, at most one per tile.
template <typename K>
int tma_grid(const mg_ctx* h, K kern, int kind, int tiles) {
  static int per_sm[6] = {0, 0, 0, 0, 0, 0};
  if (per_sm[kind] == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TM_NT, tma_smem(kind)) != cudaSuccess || b < 1) b = 1;
    cudaGetLastError();
    per_sm[kind] = b;
  }
  return std::min(tiles, h->sms * per_sm[kind]);
}

bool aligned16(const void* p, int ld) { return ((uintptr_t)p & 15) == 0 && (ld & 3) == 0; }

// Whether the tensor-copy passes take this launch: nu = 2, a large level, 16-byte aligned arrays
// with pitches of whole 16-byte units (the tensor maps' rule), the encoder available.
bool tma_pass_a_ok(const mg_ctx* h, const PassAArgs<float>& a) {
  return h->tma32 && a.nu == 2 && a.n >= TMA_MIN_N && a.vout && (a.vin == nullptr || aligned16(a.vin, a.ldvin)) &&
         aligned16(a.f, a.ldf) && aligned16(a.vout, a.ldvout) && ((uintptr_t)a.fc & 7) == 0 && (a.ldc & 1) == 0 &&
         tensor_map_encoder() != nullptr;
}
bool tma_pass_b_ok(const mg_ctx* h, const PassBArgs<float>& a) {
  return h->tma32 && a.nu == 2 && a.n >= TMA_MIN_N && a.partial == nullptr && aligned16(a.vin, a.ldvin) &&
         aligned16(a.f, a.ldf) && aligned16(a.vout, a.ldvout) && aligned16(a.vc, a.ldc) &&
         tensor_map_encoder() != nullptr;
}

TmaPassArgs tma_args(const mg_ctx* h, int kind, int n, int level, const float* coef, const int* skip, int* err) {
  TmaPassArgs t;
  t.n = n;
  t.ty = tma_ty(kind);
  t.tiles_x = (n + TM_TX - 1) / TM_TX;
  t.tiles = t.tiles_x * ((n + t.ty - 1) / t.ty);
  t.level = level;
  t.coef = coef;
  t.skip = skip;
  t.err = err;
  t.stall_tile = -1;
  t.vout = nullptr;
  t.ldvout = 0;
  t.fc = nullptr;
  t.ldc = 0;
  (void)h;
  return t;
}

int launch_pass_a_tma32(mg_ctx* h, const PassAArgs<float>& a, cudaStream_t s) {
  const int kind = tma_kind(a.vin ? TMA_A : TMA_A_ZERO, a.n);
  TmaPassArgs t = tma_args(h, kind, a.n, a.level, a.coef, a.skip, h->ints + I_ERR);
  if (a.level == 0) t.stall_tile = h->stall_tile;
  t.vout = a.vout;
  t.ldvout = a.ldvout;
  t.fc = a.fc;
  t.ldc = a.ldc;
  const int R = tm_rows_a(t.ty, 2);
  CUtensorMap mv, mf;
  KC_TRY(make_map_f32(&mf, a.f, a.n, a.n, a.ldf, TM_P, R));
  if (a.vin) KC_TRY(make_map_f32(&mv, a.vin, a.n, a.n, a.ldvin, TM_P, R));
  else mv = mf;  // not read from a zero start
  auto go = [&](auto k) { k<<<tma_grid(h, k, kind, t.tiles), TM_NT, tma_smem(kind), s>>>(mv, mf, t); };
  switch (kind) {
    case TMA_A: go(pass_a_tma32<false, TMA_TY_A>); break;
    case TMA_A_ZERO: go(pass_a_tma32<true, TMA_TY_A0>); break;
    case TMA_SMALL + TMA_A: go(pass_a_tma32<false, TMA_TY_S>); break;
    default: go(pass_a_tma32<true, TMA_TY_S>); break;
  }
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

int launch_pass_b_tma32(mg_ctx* h, const PassBArgs<float>& a, cudaStream_t s) {
  const int kind = tma_kind(TMA_B, a.n);
  TmaPassArgs t = tma_args(h, kind, a.n, a.level, a.coef, a.skip, h->ints + I_ERR);
  t.vout = a.vout;
  t.ldvout = a.ldvout;
  const int nc = (a.n - 1) / 2;
  CUtensorMap mv, mf, mc;
  KC_TRY(make_map_f32(&mv, a.vin, a.n, a.n, a.ldvin, TM_P, tm_rows_b(t.ty, 2)));
  KC_TRY(make_map_f32(&mf, a.f, a.n, a.n, a.ldf, TM_P, tm_rows_b(t.ty, 2)));
  KC_TRY(make_map_f32(&mc, a.vc, nc, nc, a.ldc, TM_CP, tm_crows_b(t.ty, 2)));
  auto go = [&](auto k) { k<<<tma_grid(h, k, kind, t.tiles), TM_NT, tma_smem(kind), s>>>(mv, mf, mc, t); };
  if (kind == TMA_B) go(pass_b_tma32<TMA_TY_B>);
  else go(pass_b_tma32<TMA_TY_S>);
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

// The coarse kernel variant for the handle: line relaxation (symmetric operators) or damped
// Jacobi on the symmetric or the general stencil.
template <typename T>
int launch_coarse(const mg_ctx* h, const CoarseArgs<T>& a, int blocks, size_t sm, cudaStream_t s) {
  if (a.ltab) {
    coarse_kernel<T, nt_coarse<T>(), true><<<blocks, nt_coarse<T>(), sm, s>>>(a);
  } else if (h->nonsym) {
    if constexpr (std::is_same<T, double>::value) {
      coarse_kernel<T, nt_coarse<T>(), false, true><<<blocks, nt_coarse<T>(), sm, s>>>(a);
    } else {
      return MG_ERR_ARG;
    }
  } else {
    coarse_kernel<T, nt_coarse<T>(), false><<<blocks, nt_coarse<T>(), sm, s>>>(a);
  }
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

// Level whose calls the coarse kernel condenses into precomputed affine maps: the side-7 level,
// when a coarser level exists (-1 otherwise, and under semi-coarsening).
int map_level(const mg_ctx* h) {
  const int d = h->k - 3;
  return (!h->semi && d >= 0 && d < h->levels - 1) ? d : -1;
}

template <typename T>
CoarseArgs<T> coarse_args(mg_ctx* h, const BindingT<T>& b, int k1, int k2, int zero1, bool adjoint,
                          const int* skip) {
  const int lc = lc_of<T>(h);
  CoarseArgs<T> a;
  a.v = lv_v(h, b, lc);
  a.f = lv_f(h, b, lc);
  a.coef = Arr<T>::coef(h);
  a.coef64 = h->coef;
  a.cinv = h->cinv;
  a.skip = skip;
  a.ldv = lv_ld(h, b, lc);
  a.ldf = lv_ld(h, b, lc);
  a.n_lc = h->lv[lc].n;
  a.lc = lc;
  a.L = h->levels;
  a.nu1 = h->nu1;
  a.nu2 = h->nu2;
  a.k1 = k1;
  a.k2 = k2;
  a.zero1 = zero1;
  a.adjoint = adjoint ? 1 : 0;
  a.ltab = h->smoother == 1 ? Arr<T>::ltab(h) : nullptr;
  a.linv = (h->smoother == 1 && std::is_same<T, double>::value) ? h->linv : nullptr;
  a.k = h->k;
  a.xonly = h->smoother == 2 ? 1 : 0;
  const int dm = map_level(h);
  a.cmap = (!adjoint && dm >= lc && Arr<T>::maps_ok(h)) ? Arr<T>::cmap(h) : nullptr;
  a.dcond = dm - lc;
  a.ncls = h->levels - dm;
  a.basis = 0;
  a.cmap_out = nullptr;
  a.map_smem = 0;
  return a;
}

// Dynamic shared memory of a coarse walk with these arguments; turns on the shared-memory copy of
// the condensed-call maps when they fit, for FP32 walks only. Measured at 4095^2: FP32 walks gain
// (mixed kappa=4 solve 904 -> 888 ms), while copying the FP64 maps (115 KB per launch) costs more
// than their reads from L2 do (FP64 kappa=4 solve 2,107 -> 2,140 ms).
template <typename T>
size_t coarse_walk_smem(const mg_ctx* h, CoarseArgs<T>& a) {
  (void)h;
  const size_t base = coarse_smem<T>(a.n_lc, a.L - a.lc);
  a.map_smem = 0;
  if (std::is_same<T, float>::value && a.cmap && base + coarse_map_smem<T>(a.ncls) <= coarse_smem_max<T>()) {
    a.map_smem = 1;
    return base + coarse_map_smem<T>(a.ncls);
  }
  return base;
}

// CTAs of a stand-alone children_kernel launch: one row of P per warp, at most two CTAs per SM, at
// least the fused call's cluster size; the cluster size in a batch, whose concurrent branches share
// the SMs.
template <typename T>
int child_parts(const mg_ctx* h, int side) {
  if (h->batched) return CHILD_PARTS;
  constexpr int NW = nt_coarse<T>() / 32;
  const int rows = side * side;
  return std::max(CHILD_PARTS, std::min((rows + NW - 1) / NW, 2 * h->sms));
}

// The condensed child-call map for calls (k1, k2) from zero at the coarse-kernel level, or nullptr
// (adjoint cycles, a nonzero start, other counter pairs, maps not built).
template <typename T>
const T* child_map(const mg_ctx* h, int k1, int k2, int zero1, bool adjoint, int* ld) {
  if (adjoint || !zero1 || lc_of<T>(h) < 1 || k2 != (k1 > 1 ? k1 - 1 : 0)) return nullptr;
  return Arr<T>::pmap(h, k1, ld);
}

template <typename T>
int emit_coarse(mg_ctx* h, const BindingT<T>& b, int k1, int k2, int zero1, bool adjoint, const int* skip,
                cudaStream_t s) {
  const int lc = lc_of<T>(h);
  CoarseArgs<T> a = coarse_args(h, b, k1, k2, zero1, adjoint, skip);
  int pld = 0;
  if (const T* pmap = child_map<T>(h, k1, k2, zero1, adjoint, &pld)) {
    prof_begin(h, K_COARSE, lc, s);
    children_kernel<T, nt_coarse<T>()><<<child_parts<T>(h, a.n_lc), nt_coarse<T>(), (size_t)pld * sizeof(T), s>>>(pmap, pld, a);
    prof_end(h, s);
    KC_CUDA(cudaGetLastError());
    ++h->launch_count;
    return MG_OK;
  }
  const size_t sm = coarse_walk_smem(h, a);
  prof_begin(h, K_COARSE, lc, s);
  KC_TRY(launch_coarse(h, a, 1, sm, s));
  prof_end(h, s);
  KC_CUDA(cudaGetLastError());
  ++h->launch_count;
  return MG_OK;
}

// The maps of condensed calls: one map-mode launch of the coarse kernel per counter class, whose
// 2 S blocks run a call at the side-7 level from each unit vector of v and of f. Runs on the
// handle's own stream outside any capture.
template <typename T>
int compute_maps(mg_ctx* h) {
  const int dm = map_level(h);
  if (dm < 0) return MG_OK;
  CoarseArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.coef = Arr<T>::coef(h);
  a.coef64 = h->coef;
  a.cinv = h->cinv;
  a.n_lc = 7;
  a.lc = dm;
  a.L = h->levels;
  a.nu1 = h->nu1;
  a.nu2 = h->nu2;
  a.k2 = 0;
  a.zero1 = 0;
  a.adjoint = 0;
  a.ltab = h->smoother != 0 ? Arr<T>::ltab(h) : nullptr;
  a.linv = (h->smoother != 0 && std::is_same<T, double>::value) ? h->linv : nullptr;
  a.k = h->k;
  a.xonly = h->smoother == 2 ? 1 : 0;
  a.cmap = nullptr;
  a.basis = 1;
  const size_t sm = coarse_smem<T>(7, h->levels - dm);
  for (int c = 1; c <= h->levels - dm; ++c) {
    a.k1 = c;
    a.cmap_out = Arr<T>::cmap(h) + (size_t)(c - 1) * 2 * MAP_S * MAP_S;
    KC_TRY(launch_coarse(h, a, 2 * MAP_S, sm, h->own));
    KC_CUDA(cudaGetLastError());
  }
  KC_CUDA(cudaStreamSynchronize(h->own));
  return MG_OK;
}

// Largest coarse-kernel side whose child calls are condensed, and the memory cap of the maps.
constexpr int PM_MAX_SIDE = 63;
constexpr size_t PM_MAX_BYTES = size_t(512) << 20;

// The condensed child-call maps P_c of the cycle in precision T (see children_matvec): for each
// class c = 1 .. levels - lc + 1, one map-mode launch of the FP64 coarse kernel at level lc whose S
// blocks run the calls (c, c - 1) from v = 0, f = e_b (FP64 arithmetic whatever T is), then a
// conversion to row-major T. Needs a coarse level below the finest one of side <= PM_MAX_SIDE.
template <typename T>
int compute_pmaps(mg_ctx* h) {
  const int lc = lc_of<T>(h);
  if (h->semi || lc < 1 || lc >= h->levels) return MG_ERR_ARG;
  const int side = h->lv[lc].n, S = side * side;
  const int cls = h->levels - lc + 1;
  const int ld = round_up(S, 16 / (int)sizeof(T));
  const size_t bytes = (size_t)cls * S * ld * sizeof(T);
  if (side > PM_MAX_SIDE || bytes > PM_MAX_BYTES) return MG_ERR_ARG;
  T*& dst = std::is_same<T, double>::value ? reinterpret_cast<T*&>(h->pm) : reinterpret_cast<T*&>(h->pm32);
  if (dst) KC_CUDA(cudaFree(dst));
  dst = nullptr;
  KC_CUDA(cudaMalloc(&dst, bytes));
  double* tmp = nullptr;
  KC_CUDA(cudaMalloc(&tmp, sizeof(double) * (size_t)S * S));
  CoarseArgs<double> a;
  memset(&a, 0, sizeof(a));
  a.coef = h->coef;
  a.coef64 = h->coef;
  a.cinv = h->cinv;
  a.n_lc = side;
  a.lc = lc;
  a.L = h->levels;
  a.nu1 = h->nu1;
  a.nu2 = h->nu2;
  a.zero1 = 1;
  a.ltab = h->smoother != 0 ? h->ltab : nullptr;
  a.linv = h->smoother != 0 ? h->linv : nullptr;
  a.k = h->k;
  a.xonly = h->smoother == 2 ? 1 : 0;
  a.basis = 2;
  a.cmap_out = tmp;
  const size_t sm = coarse_smem<double>(side, h->levels - lc);
  int st = MG_OK;
  for (int c = 1; c <= cls && st == MG_OK; ++c) {
    a.k1 = c;
    a.k2 = c > 1 ? c - 1 : 0;
    st = launch_coarse(h, a, S, sm, h->own);
    if (st == MG_OK) {
      pmap_convert_kernel<T><<<256, 256, 0, h->own>>>(tmp, S, ld, dst + (size_t)(c - 1) * S * ld);
      if (cudaGetLastError() != cudaSuccess) st = MG_ERR_CUDA;
    }
  }
  if (cudaStreamSynchronize(h->own) != cudaSuccess && st == MG_OK) st = MG_ERR_CUDA;
  cudaFree(tmp);
  if (st != MG_OK) return st;
  if (std::is_same<T, double>::value) {
    h->pm_cls = cls; h->pm_ld = ld; h->pm_side = side;
  } else {
    h->pm32_cls = cls; h->pm32_ld = ld; h->pm32_side = side;
  }
  return MG_OK;
}

// Compute whichever maps are stale (the FP32 ones only once the FP32 hierarchy exists). A
// failure leaves the flag clear: the coarse kernel then runs those calls step by step.
void ensure_maps(mg_ctx* h) {
  if (!h->maps_ok && compute_maps<double>(h) == MG_OK) h->maps_ok = true;
  if (h->have32 && !h->maps32_ok && compute_maps<float>(h) == MG_OK) h->maps32_ok = true;
  if (h->condense && !h->pm_ok && compute_pmaps<double>(h) == MG_OK) h->pm_ok = true;
  if (h->condense && h->have32 && !h->pm32_ok && compute_pmaps<float>(h) == MG_OK) h->pm32_ok = true;
  cudaGetLastError();  // a refused map leaves no sticky error: those calls run step by step
}

// With `lines` (zebra smoothing done in place by the line kernels) pass A only restricts the
// residual of the level's v: no relaxation and no copy of v.
template <typename T>
PassAArgs<T> pass_a_args(mg_ctx* h, const BindingT<T>& b, int l, bool zero, int nu, const int* skip, bool lines,
                         double* norm_partial) {
  PassAArgs<T> a;
  a.partial = norm_partial;
  a.vin = zero ? nullptr : lv_v(h, b, l);
  // lines mode from a zero start without pre-relaxation: v is written (as zero) for the post-smoothing
  a.vout = lines ? (zero ? lv_v(h, b, l) : nullptr) : Arr<T>::tmp(h, l);
  a.f = lv_f(h, b, l);
  a.fc = Arr<T>::f(h, l + 1);
  a.coef = Arr<T>::coef(h);
  a.skip = skip;
  a.ldvin = lv_ld(h, b, l);
  a.ldvout = Arr<T>::ld(h, l);
  a.ldf = lv_ld(h, b, l);
  a.ldc = Arr<T>::ld(h, l + 1);
  a.n = h->lv[l].n;
  a.nu = nu;
  a.level = l;
  return a;
}

template <typename T>
int emit_pass_a(mg_ctx* h, const BindingT<T>& b, int l, bool zero, int nu, const int* skip, cudaStream_t s,
                bool lines = false, double* norm_partial = nullptr) {
  const PassAArgs<T> a = pass_a_args(h, b, l, zero, nu, skip, lines, norm_partial);
  ++h->launch_count;
  prof_begin(h, K_PASS_A, l, s);
  int st;
  if constexpr (std::is_same<T, float>::value) {
    if (!lines && tma_pass_a_ok(h, a)) {
      st = launch_pass_a_tma32(h, a, s);
      prof_end(h, s);
      return st;
    }
    if (!lines && fast32_ok(a.n, nu, a.vin, a.ldvin) && fast32_ok(a.n, nu, a.f, a.ldf) &&
        fast32_ok(a.n, nu, a.vout, a.ldvout) &&
        ((uintptr_t)a.fc & 7) == 0 && (a.ldc & 1) == 0) {
      st = launch_pass_a_tile32(a, s);
      prof_end(h, s);
      return st;
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    const int w = (!lines && l >= 1 && !a.partial && !h->nonsym && !h->batched) ? wide_edge(a.n, h->sms) : 0;
    if (w) {
      st = w == 44 ? launch_pass_a<Tile44>(a, s) : launch_pass_a<Tile22>(a, s);
      prof_end(h, s);
      return st;
    }
  }
  switch (tile_edge(a.n)) {
    case 64: st = a.partial ? launch_pass_a<Tile64>(a, s, h->nonsym) : launch_pass_a<Tile64N>(a, s, h->nonsym); break;
    case 32: st = launch_pass_a<Tile32>(a, s, h->nonsym); break;
    case 16: st = launch_pass_a<Tile16>(a, s, h->nonsym); break;
    default: st = launch_pass_a<Tile8>(a, s, h->nonsym); break;
  }
  prof_end(h, s);
  return st;
}

// With `lines` pass B only adds the prolonged correction to the level's v, in place.
template <typename T>
PassBArgs<T> pass_b_args(mg_ctx* h, const BindingT<T>& b, int l, int nu, double* partial, const int* skip,
                         bool lines) {
  PassBArgs<T> a;
  a.vin = lines ? lv_v(h, b, l) : Arr<T>::tmp(h, l);
  a.vout = lv_v(h, b, l);
  a.f = lv_f(h, b, l);
  a.vc = Arr<T>::v(h, l + 1);
  a.coef = Arr<T>::coef(h);
  a.skip = skip;
  a.partial = partial;
  a.ldvin = Arr<T>::ld(h, l);
  a.ldvout = lv_ld(h, b, l);
  a.ldf = lv_ld(h, b, l);
  a.ldc = Arr<T>::ld(h, l + 1);
  a.n = h->lv[l].n;
  a.nu = nu;
  a.level = l;
  return a;
}

template <typename T>
int emit_pass_b(mg_ctx* h, const BindingT<T>& b, int l, int nu, double* partial, const int* skip, cudaStream_t s,
                bool lines = false) {
  const PassBArgs<T> a = pass_b_args(h, b, l, nu, partial, skip, lines);
  ++h->launch_count;
  prof_begin(h, K_PASS_B, l, s);
  int st;
  if constexpr (std::is_same<T, float>::value) {
    if (!lines && tma_pass_b_ok(h, a)) {
      st = launch_pass_b_tma32(h, a, s);
      prof_end(h, s);
      return st;
    }
    if (!lines && partial == nullptr && fast32_ok(a.n, nu, a.vin, a.ldvin) && fast32_ok(a.n, nu, a.f, a.ldf) &&
        fast32_ok(a.n, nu, a.vout, a.ldvout) && ((uintptr_t)a.vc & 7) == 0 && (a.ldc & 1) == 0) {
      st = launch_pass_b_fast32(a, s);
      prof_end(h, s);
      return st;
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    const int w = (!lines && l >= 1 && !a.partial && !h->nonsym && !h->batched) ? wide_edge(a.n, h->sms) : 0;
    if (w) {
      st = w == 44 ? launch_pass_b<Tile44>(a, s) : launch_pass_b<Tile22>(a, s);
      prof_end(h, s);
      return st;
    }
  }
  switch (tile_edge(a.n)) {
    case 64: st = a.partial ? launch_pass_b<Tile64>(a, s, h->nonsym) : launch_pass_b<Tile64N>(a, s, h->nonsym); break;
    case 32: st = launch_pass_b<Tile32>(a, s, h->nonsym); break;
    case 16: st = launch_pass_b<Tile16>(a, s, h->nonsym); break;
    default: st = launch_pass_b<Tile8>(a, s, h->nonsym); break;
  }
  prof_end(h, s);
  return st;
}

int emit_apply(mg_ctx* h, const double* v, const double* f, double* out, double* partial, const int* skip,
               cudaStream_t s) {
  const int n = h->n;
  dim3 grid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
  prof_begin(h, K_APPLY, 0, s);
  if (h->nonsym)
    apply_kernel<double, NT_VEC, true><<<grid, NT_VEC, 0, s>>>(v, f, out, h->coef, 0, n, n, partial, skip);
  else
    apply_kernel<double, NT_VEC><<<grid, NT_VEC, 0, s>>>(v, f, out, h->coef, 0, n, n, partial, skip);
  prof_end(h, s);
  KC_CUDA(cudaGetLastError());
  ++h->launch_count;
  return MG_OK;
}

// Semi-coarsened levels with at most LONG_ROWS rows of one colour: one cluster per row. (Under full
// coarsening a level has as many lines as points per line, and the segment kernel fits.)
constexpr int LONG_ROWS = 512;

template <typename T>
bool long_rows(const LineArgs<T>& a) {
  return a.semi && a.n <= 16384 && (a.nl - a.colour + 1) / 2 <= LONG_ROWS;
}

// One row per cluster of 8 CTAs of 128 threads (8 SMs per row): 1 to 16 points per thread.
constexpr int ROW_CLUSTER = 8;

template <typename T>
int launch_long_rows(const LineArgs<T>& a, cudaStream_t s) {
  const int nl = (a.nl - a.colour + 1) / 2;
  const int grid = nl * ROW_CLUSTER;
  if (a.n <= 1024) line_cluster_kernel<T, 1, 128, ROW_CLUSTER><<<grid, 128, 0, s>>>(a);
  else if (a.n <= 2048) line_cluster_kernel<T, 2, 128, ROW_CLUSTER><<<grid, 128, 0, s>>>(a);
  else if (a.n <= 4096) line_cluster_kernel<T, 4, 128, ROW_CLUSTER><<<grid, 128, 0, s>>>(a);
  else if (a.n <= 8192) line_cluster_kernel<T, 8, 128, ROW_CLUSTER><<<grid, 128, 0, s>>>(a);
  else line_cluster_kernel<T, 16, 128, ROW_CLUSTER><<<grid, 128, 0, s>>>(a);
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

template <typename T, int DIR>
int launch_lines(const LineArgs<T>& a, cudaStream_t s) {
  if (DIR == 0 && long_rows(a)) return launch_long_rows(a, s);
  const int nl = (a.nl - a.colour + 1) / 2;
  const int blocks = (nl + LINE_R - 1) / LINE_R;
  switch (line_chunk(a.n)) {
    case 16: line_relax_kernel<T, DIR, LINE_R, 16><<<blocks, 32 * LINE_R, line_smem<T, LINE_R, 16>(), s>>>(a); break;
    case 8: line_relax_kernel<T, DIR, LINE_R, 8><<<blocks, 32 * LINE_R, line_smem<T, LINE_R, 8>(), s>>>(a); break;
    case 4: line_relax_kernel<T, DIR, LINE_R, 4><<<blocks, 32 * LINE_R, line_smem<T, LINE_R, 4>(), s>>>(a); break;
    case 2: line_relax_kernel<T, DIR, LINE_R, 2><<<blocks, 32 * LINE_R, line_smem<T, LINE_R, 2>(), s>>>(a); break;
    default: line_relax_kernel<T, DIR, LINE_R, 1><<<blocks, 32 * LINE_R, line_smem<T, LINE_R, 1>(), s>>>(a); break;
  }
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

// `sweeps` zebra relaxations of level l in place: the k-th (from 0) along x for even k, along y for
// odd k, each colour 0 then colour 1. From a zero start the first half-sweep sees zero neighbours.
// With vc (post-smoothing) the first launch reads its neighbouring rows as v + P vc, which folds the
// coarse-grid correction into it: every line is then solved before its own old value is needed.
template <typename T>
int emit_lines(mg_ctx* h, const BindingT<T>& b, int l, int sweeps, bool zero, const int* skip, cudaStream_t s,
               const T* vc = nullptr, int ldc = 0) {
  LineArgs<T> a;
  a.ldc = ldc;
  a.v = lv_v(h, b, l);
  a.f = lv_f(h, b, l);
  a.coef = Arr<T>::coef(h);
  a.skip = skip;
  a.n = h->lv[l].nx;  // points per row; columns (full coarsening only) have as many
  a.nl = h->lv[l].n;
  a.ld = lv_ld(h, b, l);
  a.level = l;
  a.semi = h->semi;
  for (int k = 0; k < sweeps; ++k) {
    const int dir = h->smoother == 2 ? 0 : (k & 1);
    a.tab = Arr<T>::ltab(h) + line_tab_offset(h->k, l, dir, h->semi);
    for (int colour = 0; colour < 2; ++colour) {
      a.colour = colour;
      a.zero = (zero && k == 0 && colour == 0) ? 1 : 0;
      a.vc = (k == 0 && colour == 0) ? vc : nullptr;
      ++h->launch_count;
      prof_begin(h, dir == 0 ? K_LINES_X : K_LINES_Y, l, s);
      const int st = dir == 0 ? launch_lines<T, 0>(a, s) : launch_lines<T, 1>(a, s);
      prof_end(h, s);
      KC_TRY(st);
    }
  }
  return MG_OK;
}

// Semi-coarsening along y with x-line zebra (Section 4, solvers 5-6): every level, the coarsest
// included, runs as multi-CTA launches (the levels keep all n columns, so none is small enough for
// the single-CTA kernel). The coarsest level is one row: its x-line solve is the exact solve.
template <typename T>
int emit_call_semi(mg_ctx* h, const BindingT<T>& b, int l, int kappa, bool zero, bool norm, const int* skip,
                   cudaStream_t s) {
  const int L = h->levels;
  const int nx = h->lv[l].nx;
  if (l == L - 1) {
    LineArgs<T> a;
    a.v = lv_v(h, b, l);
    a.f = lv_f(h, b, l);
    a.coef = Arr<T>::coef(h);
    a.tab = Arr<T>::ltab(h) + line_tab_offset(h->k, l, 0, 1);
    a.skip = skip;
    a.vc = nullptr;
    a.n = nx;
    a.nl = h->lv[l].n;
    a.ld = lv_ld(h, b, l);
    a.level = l;
    a.ldc = 0;
    a.colour = 0;
    a.zero = 1;
    a.semi = 1;
    ++h->launch_count;
    prof_begin(h, K_LINES_X, l, s);
    const int st = launch_lines<T, 0>(a, s);
    prof_end(h, s);
    return st;
  }
  const int nu_pre = h->nu1, nu_post = h->nu2;
  const int nyc = h->lv[l + 1].n;
  if (nu_pre > 0) KC_TRY(emit_lines(h, b, l, nu_pre, zero, skip, s));
  {
    dim3 grid((nx + 31) / 32, (nyc + NT_VEC / 32 - 1) / (NT_VEC / 32));
    ++h->launch_count;
    prof_begin(h, K_PASS_A, l, s);
    restrict_y_kernel<T, NT_VEC><<<grid, NT_VEC, 0, s>>>(lv_v(h, b, l), lv_f(h, b, l), Arr<T>::f(h, l + 1),
                                                          Arr<T>::coef(h), l, nx, nyc, lv_ld(h, b, l),
                                                          lv_ld(h, b, l), Arr<T>::ld(h, l + 1),
                                                          (zero && nu_pre == 0) ? 1 : 0, skip);
    prof_end(h, s);
    KC_CUDA(cudaGetLastError());
  }
  if (zero && nu_pre == 0) {  // v^l = 0 before the correction is added
    KC_CUDA(cudaMemset2DAsync(lv_v(h, b, l), sizeof(T) * lv_ld(h, b, l), 0, sizeof(T) * nx, h->lv[l].n, s));
  }
  int k1 = kappa, k2 = kappa > 1 ? kappa - 1 : 0;
  KC_TRY(emit_call_semi(h, b, l + 1, k1, true, false, skip, s));
  if (k2 > 0) KC_TRY(emit_call_semi(h, b, l + 1, k2, false, false, skip, s));
  if (nu_post > 0) {
    KC_TRY(emit_lines(h, b, l, nu_post, false, skip, s, Arr<T>::v(h, l + 1), Arr<T>::ld(h, l + 1)));
  } else {
    dim3 grid((nx + 31) / 32, (h->lv[l].n + NT_VEC / 32 - 1) / (NT_VEC / 32));
    ++h->launch_count;
    prof_begin(h, K_PASS_B, l, s);
    prolong_y_add_kernel<T, NT_VEC><<<grid, NT_VEC, 0, s>>>(lv_v(h, b, l), Arr<T>::v(h, l + 1), nx, nyc,
                                                             lv_ld(h, b, l), Arr<T>::ld(h, l + 1), skip);
    prof_end(h, s);
    KC_CUDA(cudaGetLastError());
  }
  if (norm && l == 0) {
    if constexpr (std::is_same<T, double>::value) {
      KC_TRY(emit_apply(h, b.v0, b.f0, nullptr, h->partial, skip, s));
    } else {
      return MG_ERR_ARG;
    }
  }
  return MG_OK;
}

// Counters of the two coarse calls made by a call with counter kappa (Algorithm 3); the adjoint
// cycle makes them in the opposite order.
void child_counters(int kappa, bool adjoint, int* first, int* second) {
  if (!adjoint) {
    *first = kappa;
    *second = kappa > 1 ? kappa - 1 : 0;
  } else {
    *first = kappa > 1 ? kappa - 1 : kappa;
    *second = kappa > 1 ? kappa : 0;
  }
}

// emit call(l, kappa) for a fine level l < lc; `norm` adds residual partial sums at level 0
// Calls at the level just above the coarse kernel's as one cluster launch: FP64 tiles of 8 (so a
// 31^2 level has 16 CTAs, each with the FP64 work of one 8 x 8 tile), FP32 tiles of 16 (63^2: 16
// CTAs).
template <typename T>
constexpr int call_tile() { return std::is_same<T, double>::value ? 8 : 16; }

template <typename T>
int call_ctas(const mg_ctx* h, int l) {
  const int t = (h->lv[l].n + call_tile<T>() - 1) / call_tile<T>();
  return t * t;
}

// Whether the device runs the call clusters (the cluster size above 8 is non-portable); checked
// once per process and kernel variant.
template <typename T, bool NS>
bool call_cluster_supported() {
  static int ok = -1;
  if (ok < 0) {
    auto kern = call_cluster_kernel<T, nt_coarse<T>(), call_tile<T>(), NS>;
    const size_t sm = std::max(call_cluster_smem_tiles<T, call_tile<T>()>(MAX_NU, MAX_NU), coarse_smem_max<T>());
    ok = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CALL_MAX_CTAS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(CALL_MAX_CTAS);
      cfg.blockDim = dim3(nt_coarse<T>());
      cfg.dynamicSmemBytes = sm;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters >= 1) ok = 1;
    }
    cudaGetLastError();  // a refused attribute leaves no sticky error
  }
  return ok == 1;
}

// (lc: the first coarse-kernel level of the cycle in T; -1: the handle's current one)
template <typename T>
bool fused_call_ok(const mg_ctx* h, int l, bool adjoint, int lc = -1) {
  if (lc < 0) lc = lc_of<T>(h);
  if (!h->fused || adjoint || h->smoother != 0 || h->semi || l < 1 || l + 1 != lc) return false;
  if (h->nu1 > MAX_NU || h->nu2 > MAX_NU || call_ctas<T>(h, l) > CALL_MAX_CTAS) return false;
  if (h->nonsym) {
    if constexpr (std::is_same<T, double>::value) return call_cluster_supported<T, true>();
    return false;
  }
  return call_cluster_supported<T, false>();
}

template <typename T>
int emit_call_fused(mg_ctx* h, const BindingT<T>& b, int l, int kappa, bool zero, const int* skip,
                    cudaStream_t s) {
  int k1, k2;
  child_counters(kappa, false, &k1, &k2);
  const PassAArgs<T> pa = pass_a_args(h, b, l, zero, h->nu1, skip, false, nullptr);
  CoarseArgs<T> ca = coarse_args(h, b, k1, k2, 1, false, skip);
  const size_t sm_walk = coarse_walk_smem(h, ca);
  const PassBArgs<T> pb = pass_b_args(h, b, l, h->nu2, nullptr, skip, false);
  int pld = 0;
  const T* pmap = child_map<T>(h, k1, k2, 1, false, &pld);
  constexpr int NT = nt_coarse<T>(), TILE = call_tile<T>();
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = call_ctas<T>(h, l);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(call_ctas<T>(h, l));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = std::max(call_cluster_smem_tiles<T, TILE>(h->nu1, h->nu2), sm_walk);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++h->launch_count;
  prof_begin(h, K_CALL, l, s);
  if constexpr (std::is_same<T, double>::value) {
    if (h->nonsym) {
      KC_CUDA(cudaLaunchKernelEx(&cfg, call_cluster_kernel<T, NT, TILE, true>, pa, ca, pb, pmap, pld));
    } else {
      KC_CUDA(cudaLaunchKernelEx(&cfg, call_cluster_kernel<T, NT, TILE, false>, pa, ca, pb, pmap, pld));
    }
  } else {
    KC_CUDA(cudaLaunchKernelEx(&cfg, call_cluster_kernel<T, NT, TILE, false>, pa, ca, pb, pmap, pld));
  }
  prof_end(h, s);
  return MG_OK;
}

// Two-level fused calls (call2_cluster_kernel): a call two levels above the coarse kernel's with its
// child calls, whose own children are condensed. Tiles of 32 (FP32) / 16 (FP64) at that level, so a
// 127^2 (FP32) or 63^2 (FP64) level has 16 of them, one per CTA of the cluster.
template <typename T>
constexpr int call2_tile() { return std::is_same<T, double>::value ? 16 : 32; }

template <typename T>
bool call2_cluster_supported() {
  static int ok = -1;
  if (ok < 0) {
    auto kern = call2_cluster_kernel<T, nt_coarse<T>(), call2_tile<T>(), call_tile<T>()>;
    const size_t sm = call2_smem<T, call2_tile<T>(), call_tile<T>()>(MAX_NU, MAX_NU);
    ok = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CALL_MAX_CTAS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(CALL_MAX_CTAS);
      cfg.blockDim = dim3(nt_coarse<T>());
      cfg.dynamicSmemBytes = sm;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters >= 1) ok = 1;
    }
    cudaGetLastError();
  }
  return ok == 1;
}

template <typename T>
bool fused2_ok(const mg_ctx* h, int l, int kappa, bool adjoint) {
  const int lc = lc_of<T>(h);
  if (h->fused < 2 || adjoint || h->smoother != 0 || h->semi || h->nonsym || l < 1 || l + 2 != lc) return false;
  if (h->nu1 > MAX_NU || h->nu2 > MAX_NU) return false;
  const int t1 = (h->lv[l].n + call2_tile<T>() - 1) / call2_tile<T>();
  if (t1 * t1 > CALL_MAX_CTAS || call_ctas<T>(h, l + 1) > CALL_MAX_CTAS) return false;
  int k1, k2, ld = 0;
  child_counters(kappa, false, &k1, &k2);
  for (int c : {k1, k2}) {  // the grandchildren of each child call must be condensed
    if (c == 0) continue;
    int g1, g2;
    child_counters(c, false, &g1, &g2);
    if (!child_map<T>(h, g1, g2, 1, false, &ld)) return false;
  }
  return call2_cluster_supported<T>();
}

template <typename T>
int emit_call_fused2(mg_ctx* h, const BindingT<T>& b, int l, int kappa, bool zero, const int* skip, cudaStream_t s) {
  Call2Args<T> a;
  a.pa1 = pass_a_args(h, b, l, zero, h->nu1, skip, false, nullptr);
  a.pb1 = pass_b_args(h, b, l, h->nu2, nullptr, skip, false);
  a.pa2[0] = pass_a_args(h, b, l + 1, true, h->nu1, skip, false, nullptr);
  a.pa2[1] = pass_a_args(h, b, l + 1, false, h->nu1, skip, false, nullptr);
  a.pb2 = pass_b_args(h, b, l + 1, h->nu2, nullptr, skip, false);
  int k1, k2;
  child_counters(kappa, false, &k1, &k2);
  a.children = k2 > 0 ? 2 : 1;
  a.cc = coarse_args(h, b, 1, 0, 1, false, skip);  // v, f, pitches and side of level l + 2
  const int ks[2] = {k1, k2};
  for (int c = 0; c < 2; ++c) {
    a.pmap[c] = nullptr;
    if (ks[c] == 0) continue;
    int g1, g2;
    child_counters(ks[c], false, &g1, &g2);
    a.pmap[c] = child_map<T>(h, g1, g2, 1, false, &a.pld);
  }
  constexpr int NT = nt_coarse<T>();
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CALL_MAX_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CALL_MAX_CTAS);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = std::max(call2_smem<T, call2_tile<T>(), call_tile<T>()>(h->nu1, h->nu2),
                                  (size_t)a.pld * sizeof(T));
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++h->launch_count;
  prof_begin(h, K_CALL, l, s);
  KC_CUDA(cudaLaunchKernelEx(&cfg, call2_cluster_kernel<T, NT, call2_tile<T>(), call_tile<T>()>, a));
  prof_end(h, s);
  return MG_OK;
}

// ------------------------------------------------------------------------------------------
// Persistent deep calls (deep.cuh): a call at a side <= deep_n with everything below it in one
// cooperative launch, its child calls at the coarse-kernel level condensed.
// ------------------------------------------------------------------------------------------
constexpr int DEEP_MAX_SIDE = 511;  // tiles up to 32 x 32, as tile_edge gives up to that side

// Dynamic shared memory of a deep launch: the largest tile pass of its levels, and P's staged f.
template <typename T>
size_t deep_smem_tiles(int edge, int nu1, int nu2) {
  switch (edge) {
    case 32: return std::max(pass_a_smem<T, 32, 32>(nu1), pass_b_smem<T, 32, 32>(nu2, false));
    case 16: return std::max(pass_a_smem<T, 16, 16>(nu1), pass_b_smem<T, 16, 16>(nu2, false));
    default: return std::max(pass_a_smem<T, 8, 8>(nu1), pass_b_smem<T, 8, 8>(nu2, false));
  }
}
// Whether a deep launch from level l runs the last child's pass B inside its parent's: at least
// two levels of passes, the parent level's tiles 8 x 8, two post-sweeps, no residual sums.
template <typename T>
bool deep_merge_b(const mg_ctx* h, int l) {
  const int lc = lc_of<T>(h);
  return lc - l >= 2 && h->nu2 == 2 && tile_edge(h->lv[lc - 2].n) == 8;
}

// Whether a deep launch from level l runs a first child's pass B and the second child's pass A
// (the level above the condensed one) as one phase: that level's tiles 8 x 8, two sweeps each way,
// FP32 only (measured at 4095^2: mixed kappa=4 solve 510 -> 506 ms; in FP64 the 15 x 15 window's
// redundant FP64 work costs more than the phase it saves, 1,704 -> 1,727 ms).
template <typename T>
bool deep_merge_ba(const mg_ctx* h, int l) {
  const int lc = lc_of<T>(h);
  return std::is_same<T, float>::value && lc - l >= 2 && h->nu1 == 2 && h->nu2 == 2 &&
         tile_edge(h->lv[lc - 1].n) == 8;
}

// Launch shape of a deep launch whose top call is at level l: CTAs (two per SM where they fit,
// else one), dynamic shared memory (the tile passes and P's staged f, then each CTA's rows of P
// and their copy barrier) and the offset of those rows; false where no shape fits (a device
// without cooperative launches, or rows too many for shared memory).
struct DeepShape {
  int grid;
  size_t smem, prow_off;
  int staged;  // 0: P's rows too many for shared memory, read from global memory
};
template <typename T>
bool deep_shape(const mg_ctx* h, int l, DeepShape* out) {
  static int coop = -1;
  if (coop < 0) {
    int dev = 0, c = 0;
    coop = (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && c &&
            cudaFuncSetAttribute(deep_kernel<T, NT_DEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_CAP) == cudaSuccess)
               ? 1
               : 0;
    cudaGetLastError();
  }
  const int lc = lc_of<T>(h);
  int pld = 0;
  if (!coop || l < 1 || l >= lc || !Arr<T>::pmap(h, 1, &pld)) return false;
  size_t base = (size_t)pld * sizeof(T);
  for (int q = l; q < lc; ++q) base = std::max(base, deep_smem_tiles<T>(tile_edge(h->lv[q].n), h->nu1, h->nu2));
  if (deep_merge_b<T>(h, l)) base = std::max(base, deep_b2_smem<T>());
  if (deep_merge_ba<T>(h, l)) base = std::max(base, deep_ba_smem<T>());
  const int S = h->lv[lc].n * h->lv[lc].n;
  for (int staged = 1; staged >= 0; --staged)
    for (int per_sm = 2; per_sm >= 1; --per_sm) {
      const int grid = per_sm * h->sms;
      const size_t rows = (size_t)(S + grid - 1) / grid;
      const size_t off = (base + 15) & ~(size_t)15;
      const size_t sm = staged ? off + ((rows * pld * sizeof(T) + 15) & ~(size_t)15) + 16 : off;
      int occ = 0;
      if (sm > SMEM_CAP ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, deep_kernel<T, NT_DEEP>, NT_DEEP, sm) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (occ >= per_sm) {
        *out = DeepShape{grid, sm, off, staged};
        return true;
      }
    }
  return false;
}

// Whether the call at level l starts a deep launch: the largest level at or below deep_n, damped
// Jacobi with full coarsening and the symmetric stencil, its condensed child-call maps available.
template <typename T>
bool deep_ok(const mg_ctx* h, int l, bool adjoint) {
  const int lc = lc_of<T>(h);
  if (!h->deep_n || h->batched || adjoint || h->smoother != 0 || h->semi || h->nonsym || l < 1 || l >= lc)
    return false;
  if (h->lv[l].n > std::min(h->deep_n, DEEP_MAX_SIDE) || lc - l > DEEP_MAX_DEPTH) return false;
  if (h->nu1 > MAX_NU || h->nu2 > MAX_NU) return false;
  DeepShape sh;
  return deep_shape<T>(h, l, &sh);
}

template <typename T>
int emit_deep(mg_ctx* h, const BindingT<T>& b, int l, int kappa, bool zero, const int* skip, cudaStream_t s) {
  const int lc = lc_of<T>(h);
  DeepArgs<T> a;
  memset(&a, 0, sizeof(a));
  DeepShape sh;
  if (!deep_shape<T>(h, l, &sh)) return MG_ERR_ARG;
  for (int d = 0; d < lc - l; ++d) {
    a.pa[d] = pass_a_args(h, b, l + d, false, h->nu1, skip, false, nullptr);
    a.pb[d] = pass_b_args(h, b, l + d, h->nu2, nullptr, skip, false);
    a.tile[d] = tile_edge(h->lv[l + d].n);
  }
  a.cc = coarse_args(h, b, kappa, kappa > 1 ? kappa - 1 : 0, 1, false, skip);
  a.pmap = Arr<T>::pmap(h, 1, &a.pld);
  const int side = h->lv[lc].n;
  a.pstride = (size_t)side * side * a.pld;
  a.pcls = std::is_same<T, double>::value ? h->pm_cls : h->pm32_cls;
  a.top = l;
  a.depth = lc - l;
  a.kappa = kappa;
  a.zero = zero ? 1 : 0;
  a.bar = reinterpret_cast<unsigned*>(h->ints + I_BAR);
  a.err = h->ints + I_ERR;
  a.skip = skip;
  a.prow_off = (int)sh.prow_off;
  a.staged = sh.staged;
  a.stall_cta = h->stall_cta;
  a.merge_b = deep_merge_b<T>(h, l) ? 1 : 0;
  a.merge_ba = deep_merge_ba<T>(h, l) ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(sh.grid);
  cfg.blockDim = dim3(NT_DEEP);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++h->launch_count;
  prof_begin(h, K_DEEP, l, s);
  KC_CUDA(cudaLaunchKernelEx(&cfg, deep_kernel<T, NT_DEEP>, a));
  prof_end(h, s);
  return MG_OK;
}

template <typename T>
int emit_call(mg_ctx* h, const BindingT<T>& b, int l, int kappa, bool zero, bool adjoint, bool norm,
              const int* skip, cudaStream_t s) {
  if (deep_ok<T>(h, l, adjoint)) return emit_deep(h, b, l, kappa, zero, skip, s);
  if (fused2_ok<T>(h, l, kappa, adjoint)) return emit_call_fused2(h, b, l, kappa, zero, skip, s);
  if (fused_call_ok<T>(h, l, adjoint)) return emit_call_fused(h, b, l, kappa, zero, skip, s);
  const int nu_pre = adjoint ? h->nu2 : h->nu1;
  const int nu_post = adjoint ? h->nu1 : h->nu2;
  const bool lines = h->smoother == 1;
  if (lines && nu_pre > 0) {
    KC_TRY(emit_lines(h, b, l, nu_pre, zero, skip, s));
    KC_TRY(emit_pass_a(h, b, l, false, 0, skip, s, true));
  } else {
    KC_TRY(emit_pass_a(h, b, l, zero, lines ? 0 : nu_pre, skip, s, lines));
  }
  int k1, k2;
  child_counters(kappa, adjoint, &k1, &k2);
  if (l + 1 >= lc_of<T>(h)) {
    KC_TRY(emit_coarse(h, b, k1, k2, 1, adjoint, skip, s));
  } else {
    KC_TRY(emit_call(h, b, l + 1, k1, true, adjoint, false, skip, s));
    if (k2 > 0) KC_TRY(emit_call(h, b, l + 1, k2, false, adjoint, false, skip, s));
  }
  if (!lines) return emit_pass_b(h, b, l, nu_post, norm && l == 0 ? h->partial : nullptr, skip, s);
  if (nu_post > 0) {
    KC_TRY(emit_lines(h, b, l, nu_post, false, skip, s, Arr<T>::v(h, l + 1), Arr<T>::ld(h, l + 1)));
  } else {
    KC_TRY(emit_pass_b(h, b, l, 0, nullptr, skip, s, true));
  }
  if (norm && l == 0) {
    if constexpr (std::is_same<T, double>::value) {
      KC_TRY(emit_apply(h, b.v0, b.f0, nullptr, h->partial, skip, s));
    } else {
      return MG_ERR_ARG;
    }
  }
  return MG_OK;
}


// One finest-level cycle. With norm (FP64 only), the last pass writes residual partial sums (or,
// when the coarse kernel handles level 0, a separate residual pass does).
template <typename T>
int emit_cycle(mg_ctx* h, const BindingT<T>& b, int kappa, bool zero, bool adjoint, bool norm, const int* skip,
               cudaStream_t s) {
  if (h->semi) return emit_call_semi(h, b, 0, kappa, zero, norm, skip, s);
  if (lc_of<T>(h) == 0) {
    KC_TRY(emit_coarse(h, b, kappa, 0, zero ? 1 : 0, adjoint, skip, s));
    if (norm) {
      if constexpr (std::is_same<T, double>::value) {
        KC_TRY(emit_apply(h, b.v0, b.f0, nullptr, h->partial, skip, s));
      } else {
        return MG_ERR_ARG;
      }
    }
    return MG_OK;
  }
  return emit_call(h, b, 0, kappa, zero, adjoint, norm, skip, s);
}

// A stand-alone solve cycle whose stopping test comes first: pass A at level 0 forms the residual
// of the incoming iterate in its first sweep (the residual form of the same update) and writes its
// squares; finish_step (pre mode) records it as the residual after the previous cycle and stops
// there, skipping the rest of the cycle, or lets the cycle run. This drops the separate residual
// stage of pass B at level 0 (10 FP64 operations per point per cycle) for one extra pass A when
// the solve ends. Used for FP64 damped Jacobi with full coarsening, nu1 >= 1 and a fine level
// above the coarse kernel.
bool prenorm_ok(const mg_ctx* h) { return h->smoother == 0 && !h->semi && h->lc > 0 && h->nu1 >= 1; }

// (finish = false: the same launches without the stopping test, for per-launch profiling)
int emit_solve_cycle_prenorm(mg_ctx* h, const Binding& b, int kappa, cudaGraphConditionalHandle ch,
                             const int* skip, cudaStream_t s, bool finish = true) {
  KC_TRY(emit_pass_a(h, b, 0, false, h->nu1, skip, s, false, h->partial));
  if (finish) {
    finish_step_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(h->partial, (int)pass_grid_blocks(h->n), h->scal, h->ints,
                                                     h->hist, ch, 1, 1);
    KC_CUDA(cudaGetLastError());
    ++h->launch_count;
  }
  int k1, k2;
  child_counters(kappa, false, &k1, &k2);
  if (1 >= h->lc) {
    KC_TRY(emit_coarse(h, b, k1, k2, 1, false, skip, s));
  } else {
    KC_TRY(emit_call(h, b, 1, k1, true, false, false, skip, s));
    if (k2 > 0) KC_TRY(emit_call(h, b, 1, k2, false, false, false, skip, s));
  }
  return emit_pass_b(h, b, 0, h->nu2, nullptr, skip, s);
}

int norm_partials(mg_ctx* h) {
  return (int)((h->lc == 0 || h->smoother != 0) ? apply_grid_blocks(h->n) : pass_grid_blocks(h->n));
}

// ------------------------------------------------------------------------------------------
// Graph cache
// ------------------------------------------------------------------------------------------
GraphEntry* find_graph(mg_ctx* h, int kind, int kappa, int flag, const void* p0, const void* p1) {
  for (auto& g : h->graphs)
    if (g.kind == kind && g.kappa == kappa && g.flag == flag && g.p0 == p0 && g.p1 == p1) return &g;
  return nullptr;
}

void drop_graphs(mg_ctx* h) {
  for (auto& g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  h->graphs.clear();
}

GraphEntry* add_graph(mg_ctx* h, const GraphEntry& e) {
  h->graphs.push_back(e);
  return &h->graphs.back();
}

// Bounded cache: forget the oldest graphs. Called only at the start of a public entry point, so
// no GraphEntry pointer held by a caller inside the library is invalidated.
void ensure_maps(mg_ctx* h);

void trim_graphs(mg_ctx* h) {
  ensure_maps(h);
  while (h->graphs.size() > 24) {
    auto& g = h->graphs.front();
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    h->graphs.pop_front();
  }
}

// Plain cycle graph: flag bit0 = zero start, bit1 = adjoint.
int get_cycle_graph(mg_ctx* h, double* v, const double* f, int kappa, int flag, GraphEntry** out) {
  if ((*out = find_graph(h, G_CYCLE, kappa, flag, v, f))) return MG_OK;
  Binding b{v, f, h->n};
  cudaGraph_t g;
  h->launch_count = 0;
  KC_CUDA(cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal));
  const int st = emit_cycle(h, b, kappa, flag & 1, (flag & 2) != 0, false, nullptr, h->own);
  const cudaError_t ce = cudaStreamEndCapture(h->own, &g);
  if (st < 0) {
    if (ce == cudaSuccess) cudaGraphDestroy(g);
    return st;
  }
  KC_CUDA(ce);
  GraphEntry e;
  e.kind = G_CYCLE; e.kappa = kappa; e.flag = flag; e.p0 = v; e.p1 = f; e.graph = g;
  e.launches = h->launch_count;
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    KC_CUDA(ie);
  }
  h->last_launches = e.launches;
  *out = add_graph(h, e);
  return MG_OK;
}

// WHILE-loop graph whose body is captured from `body(handle)`.
template <typename Body>
int build_while_graph(mg_ctx* h, Body body, cudaGraph_t* g_out, cudaGraphExec_t* e_out) {
  cudaGraph_t g;
  KC_CUDA(cudaGraphCreate(&g, 0));
  auto fail = [&](cudaError_t e) {
    cudaGraphDestroy(g);
    snprintf(g_err, sizeof(g_err), "while-graph: %s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  };
  cudaGraphConditionalHandle ch;
  cudaError_t e1 = cudaGraphConditionalHandleCreate(&ch, g, 1, cudaGraphCondAssignDefault);
  if (e1 != cudaSuccess) return fail(e1);
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = ch;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e1 = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e1 != cudaSuccess) return fail(e1);
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  e1 = cudaStreamBeginCaptureToGraph(h->own, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e1 != cudaSuccess) return fail(e1);
  h->launch_count = 0;
  const int st = body(ch);
  cudaGraph_t captured;
  const cudaError_t ce = cudaStreamEndCapture(h->own, &captured);
  if (st < 0) {
    cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) return fail(ce);
  cudaGraphExec_t ex;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  if (ie != cudaSuccess) return fail(ie);
  *g_out = g;
  *e_out = ex;
  return MG_OK;
}

int ensure_hist(mg_ctx* h, int count) {
  if (count <= h->hist_cap) return MG_OK;
  if (h->hist) KC_CUDA(cudaFree(h->hist));
  h->hist = nullptr;
  h->hist_cap = 0;
  KC_CUDA(cudaMalloc(&h->hist, sizeof(double) * (size_t)count));
  h->hist_cap = count;
  // history buffer moved: graphs that write it are stale
  drop_graphs(h);
  return MG_OK;
}

int launch_norm2(mg_ctx* h, const double* x, double* out_scalar, cudaStream_t s) {
  const size_t len = (size_t)h->n * h->n;
  dot_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, s>>>(x, x, nullptr, len, h->partial2, nullptr, nullptr);
  KC_CUDA(cudaGetLastError());
  sum_to_scalar_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(h->partial2, VEC_BLOCKS, out_scalar);
  KC_CUDA(cudaGetLastError());
  return MG_OK;
}

bool valid_handle(mg_handle h) { return h && h->ok; }

// A kernel whose bounded wait (for a tensor copy, or at a deep call's grid barrier) ran out left
// its code in the error slot: report it once (MG_ERR_TIMEOUT) and clear the slot.
int device_error(mg_ctx* h, int code, cudaStream_t s) {
  if (code == 0) return MG_OK;
  // the error slot and the grid barrier's words (a timed-out barrier leaves its count behind)
  KC_CUDA(cudaMemsetAsync(h->ints + I_ERR, 0, sizeof(int) * 3, s));
  KC_CUDA(cudaStreamSynchronize(s));
  snprintf(g_err, sizeof(g_err), "%s (code %d)",
           code == DEEP_ERR_TIMEOUT ? "a persistent deep call gave up waiting at a grid barrier"
                                    : "a level kernel gave up waiting for its tensor copies",
           code);
  return MG_ERR_TIMEOUT;
}

int read_result(mg_ctx* h, cudaStream_t s, double tol, int* count_out, double* final_relres, double* history) {
  int ints[NINT];
  double scal[NSCAL];
  KC_CUDA(cudaMemcpyAsync(ints, h->ints, sizeof(ints), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaMemcpyAsync(scal, h->scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  KC_TRY(device_error(h, ints[I_ERR], s));
  const int count = ints[I_COUNT];
  if (history && count > 0) KC_CUDA(cudaMemcpy(history, h->hist, sizeof(double) * count, cudaMemcpyDeviceToHost));
  if (count_out) *count_out = count;
  if (final_relres) *final_relres = scal[S_LAST];
  return scal[S_LAST] <= tol ? MG_OK : MG_NOT_CONVERGED;
}

// Add to `parent` one instance's whole solve: a child graph with its initialisation (||f||^2,
// reset of the device state, and for the mixed form the first FP64 residual), then a WHILE
// conditional node repeating {cycle, [x += d, r = f - A x,] stopping test}.
int add_solve_branch(mg_ctx* h, cudaGraph_t parent, double* x, const double* f, int kappa, double tol, int max_iters,
                     bool mixed) {
  const int n = h->n;
  float* d = h->lv[0].v32;
  float* r32 = h->lv[0].f32;
  const int napply = (int)apply_grid_blocks(n);
  dim3 agrid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
  cudaGraph_t init;
  KC_CUDA(cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal));
  int st = launch_norm2(h, f, h->scal + S_FNORM2, h->own);
  reset_state_kernel<<<1, 1, 0, h->own>>>(h->ints, max_iters, h->scal, tol);
  if (mixed)
    ir_residual_kernel<NT_VEC><<<agrid, NT_VEC, 0, h->own>>>(x, f, r32, h->ld32_0, h->coef, n, h->partial, nullptr);
  const cudaError_t le = cudaGetLastError();
  const cudaError_t ce = cudaStreamEndCapture(h->own, &init);
  if (st < 0) return st;
  KC_CUDA(le);
  KC_CUDA(ce);
  cudaGraphNode_t init_node;
  const cudaError_t ae = cudaGraphAddChildGraphNode(&init_node, parent, nullptr, 0, init);
  cudaGraphDestroy(init);  // the child node holds its own copy
  KC_CUDA(ae);
  cudaGraphConditionalHandle ch;
  KC_CUDA(cudaGraphConditionalHandleCreate(&ch, parent, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = ch;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  KC_CUDA(cudaGraphAddNode(&node, parent, &init_node, nullptr, 1, &np));
  KC_CUDA(cudaStreamBeginCaptureToGraph(h->own, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  const int* done = h->ints + I_DONE;
  if (mixed) {
    BindingT<float> b{d, r32, h->ld32_0};
    st = emit_cycle(h, b, kappa, true, false, false, done, h->own);
    ir_add_kernel<NT_VEC><<<agrid, NT_VEC, 0, h->own>>>(x, d, n, h->ld32_0, done);
    ir_residual_kernel<NT_VEC><<<agrid, NT_VEC, 0, h->own>>>(x, f, r32, h->ld32_0, h->coef, n, h->partial, done);
    finish_step_kernel<NT_VEC><<<1, NT_VEC, 0, h->own>>>(h->partial, napply, h->scal, h->ints, h->hist, ch, 1);
  } else if (prenorm_ok(h)) {
    Binding b{x, f, n};
    st = emit_solve_cycle_prenorm(h, b, kappa, ch, done, h->own);
  } else {
    Binding b{x, f, n};
    st = emit_cycle(h, b, kappa, false, false, true, done, h->own);
    finish_step_kernel<NT_VEC><<<1, NT_VEC, 0, h->own>>>(h->partial, norm_partials(h), h->scal, h->ints, h->hist,
                                                         ch, 1);
  }
  const cudaError_t le2 = cudaGetLastError();
  cudaGraph_t captured;
  const cudaError_t ce2 = cudaStreamEndCapture(h->own, &captured);
  if (st < 0) return st;
  KC_CUDA(le2);
  KC_CUDA(ce2);
  return MG_OK;
}

int solve_impl(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles, int* cycles,
               double* final_relres, double* history, bool adjoint = false) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !f || kappa < 1 || !(tol > 0) || max_cycles < 1) return MG_ERR_ARG;
  if (adjoint && (h->smoother != 0 || h->nonsym)) return MG_ERR_ARG;
  trim_graphs(h);
  KC_TRY(ensure_hist(h, max_cycles));
  cudaStream_t s = h->stream();
  const int gflag = (adjoint ? 1 : 0) | (h->stop_rule << 1);
  GraphEntry* ge = find_graph(h, G_SOLVE, kappa, gflag, v, f);
  if (!ge) {
    GraphEntry e;
    e.kind = G_SOLVE; e.kappa = kappa; e.flag = gflag; e.p0 = v; e.p1 = f;
    Binding b{v, f, h->n};
    const int np = norm_partials(h);
    const bool err_rule = h->stop_rule == 1;
    const bool pre = !adjoint && !err_rule && prenorm_ok(h);
    KC_TRY(build_while_graph(h, [&](cudaGraphConditionalHandle ch) -> int {
      if (pre) return emit_solve_cycle_prenorm(h, b, kappa, ch, h->ints + I_DONE, h->own);
      KC_TRY(emit_cycle(h, b, kappa, false, adjoint, !err_rule, h->ints + I_DONE, h->own));
      if (err_rule) {  // ||v_k||^2 partial sums
        dot_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, h->own>>>(v, v, nullptr, (size_t)h->n * h->n, h->partial,
                                                              nullptr, h->ints + I_DONE);
        ++h->launch_count;
      }
      finish_step_kernel<NT_VEC><<<1, NT_VEC, 0, h->own>>>(h->partial, err_rule ? VEC_BLOCKS : np, h->scal, h->ints,
                                                           h->hist, ch, 1);
      KC_CUDA(cudaGetLastError());
      ++h->launch_count;
      return MG_OK;
    }, &e.graph, &e.exec));
    e.launches = h->launch_count;
    ge = add_graph(h, e);
  }
  KC_TRY(launch_norm2(h, h->stop_rule == 1 ? v : f, h->scal + S_FNORM2, s));
  reset_state_kernel<<<1, 1, 0, s>>>(h->ints, max_cycles, h->scal, tol);
  KC_CUDA(cudaGetLastError());
  KC_CUDA(cudaGraphLaunch(ge->exec, s));
  return read_result(h, s, tol, cycles, final_relres, history);
}

// Level shapes: rows 2^(k-l) - 1; columns the same (full coarsening) or n at every level (semi).
void set_geometry(mg_ctx* h) {
  for (int l = 0; l < h->levels; ++l) {
    h->lv[l].n = (1 << (h->k - l)) - 1;
    h->lv[l].nx = h->semi ? h->n : h->lv[l].n;
    h->lv[l].ld = l == 0 ? h->n : round_up(h->lv[l].nx, 32);
  }
}

int alloc_levels(mg_ctx* h) {
  set_geometry(h);
  if (h->semi) {  // in-place line relaxation everywhere: v and f per coarse level, no temporaries
    h->lc = h->levels;
    for (int l = 1; l < h->levels; ++l) {
      Level& L = h->lv[l];
      const size_t bytes = sizeof(double) * (size_t)L.ld * L.n;
      KC_CUDA(cudaMalloc(&L.v, bytes));
      KC_CUDA(cudaMalloc(&L.f, bytes));
      KC_CUDA(cudaMemsetAsync(L.v, 0, bytes, h->own));
      KC_CUDA(cudaMemsetAsync(L.f, 0, bytes, h->own));
    }
    return MG_OK;
  }
  // coarse-kernel levels: the first level whose side is <= coarse_n (at least the coarsest)
  h->lc = h->levels - 1;
  for (int l = 0; l < h->levels; ++l)
    if (h->lv[l].n <= h->coarse_n) {
      h->lc = l;
      break;
    }
  for (int l = 0; l < h->levels; ++l) {
    Level& L = h->lv[l];
    const size_t bytes = sizeof(double) * (size_t)L.ld * L.n;
    if (l < h->lc) KC_CUDA(cudaMalloc(&L.tmp, bytes));
    if (l > 0 && l <= h->lc) {
      KC_CUDA(cudaMalloc(&L.v, bytes));
      KC_CUDA(cudaMalloc(&L.f, bytes));
      KC_CUDA(cudaMemsetAsync(L.v, 0, bytes, h->own));
      KC_CUDA(cudaMemsetAsync(L.f, 0, bytes, h->own));
    }
  }
  return MG_OK;
}

// FP32 hierarchy of the mixed cycle: same shapes as the FP64 one, plus level 0 (d and r32).
int ensure_levels32(mg_ctx* h) {
  if (h->semi || h->nonsym) return MG_ERR_ARG;  // the FP32 cycles: full coarsening, symmetric operators
  if (h->have32) return MG_OK;
  h->lc32 = h->levels - 1;
  for (int l = 0; l < h->levels; ++l)
    if (h->lv[l].n <= h->coarse_n32) {
      h->lc32 = l;
      break;
    }
  h->ld32_0 = round_up(h->n, 32);
  for (int l = 0; l < h->levels; ++l) {
    Level& L = h->lv[l];
    const size_t bytes = sizeof(float) * (size_t)(l == 0 ? h->ld32_0 : L.ld) * L.n;
    if (l < h->lc32) KC_CUDA(cudaMalloc(&L.tmp32, bytes));
    if (l <= h->lc32) {
      KC_CUDA(cudaMalloc(&L.v32, bytes));
      KC_CUDA(cudaMalloc(&L.f32, bytes));
      KC_CUDA(cudaMemsetAsync(L.v32, 0, bytes, h->own));
      KC_CUDA(cudaMemsetAsync(L.f32, 0, bytes, h->own));
    }
  }
  KC_CUDA(cudaStreamSynchronize(h->own));
  h->have32 = true;
  ensure_maps(h);
  return MG_OK;
}

int free_levels(mg_ctx* h) {
  for (int l = 0; l < MAXL; ++l) {
    float** f32s[] = {&h->lv[l].v32, &h->lv[l].tmp32, &h->lv[l].f32};
    for (float** p : f32s) {
      if (*p) KC_CUDA(cudaFree(*p));
      *p = nullptr;
    }
    if (l > 0) {
      if (h->lv[l].v) KC_CUDA(cudaFree(h->lv[l].v));
      if (h->lv[l].f) KC_CUDA(cudaFree(h->lv[l].f));
      h->lv[l].v = h->lv[l].f = nullptr;
    }
    if (h->lv[l].tmp) KC_CUDA(cudaFree(h->lv[l].tmp));
    h->lv[l].tmp = nullptr;
  }
  h->have32 = false;
  h->pm_ok = h->pm32_ok = false;  // the coarse-kernel level may move
  return MG_OK;
}

int run_setup_kernels(mg_ctx* h) {
  h->maps_ok = h->maps32_ok = false;
  h->pm_ok = h->pm32_ok = false;
  setup_stencils_kernel<<<1, 32, 0, h->own>>>(h->theta, h->eps, h->n, h->levels, h->omega, h->coef, h->coef32,
                                             h->stencils, h->dstencil, h->rediscretized, h->semi, h->bx, h->by);
  KC_CUDA(cudaGetLastError());
  line_tables_kernel<<<1, 32, 0, h->own>>>(h->coef, h->k, h->levels, h->ltab, h->ltab32, h->linv, h->semi);
  KC_CUDA(cudaGetLastError());
  const int nc = h->lv[h->levels - 1].n;
  if (nc > 1 && !h->semi) {
    coarsest_inverse_kernel<<<1, 256, 0, h->own>>>(h->stencils, h->levels - 1, nc, h->work, h->cinv, h->cinv32);
    KC_CUDA(cudaGetLastError());
  }
  KC_CUDA(cudaStreamSynchronize(h->own));
  return MG_OK;
}

}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

const char* mg_status_string(int status) {
  switch (status) {
    case MG_OK: return "ok";
    case MG_NOT_CONVERGED: return "not converged within the iteration limit";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_NOMEM: return "device allocation failed";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_TIMEOUT: return "device-side wait timed out";
    case MG_ERR_STATE: return "invalid handle";
    default: return "unknown status";
  }
}

const char* mg_last_error(void) { return g_err; }

int mg_destroy(mg_handle h) {
  if (!h) return MG_OK;
  if (h->own) cudaStreamSynchronize(h->own);
  drop_graphs(h);
  free_levels(h);
  void* ptrs[] = {h->cmap, h->cmap32, h->pm, h->pm32, h->pw, h->pz2, h->coef, h->coef32, h->stencils, h->dstencil, h->ltab, h->ltab32, h->linv, h->cinv, h->cinv32, h->work, h->partial,
                  h->partial2, h->scal, h->ints, h->hist, h->pr, h->pp, h->pq, h->pz, h->pzold, h->hv, h->hf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->own) cudaStreamDestroy(h->own);
  h->ok = false;
  delete h;
  return MG_OK;
}

int mg_setup(int n, double eps, double theta, int levels, int nu1, int nu2, mg_handle* out) {
  if (!out) return MG_ERR_ARG;
  *out = nullptr;
  int k = 0;
  while (k < 15 && ((1 << k) - 1) < n) ++k;
  if (n < 1 || ((1 << k) - 1) != n || k > 14) return MG_ERR_ARG;
  if (levels < 1 || levels > k || (k - levels + 1) > 4) return MG_ERR_ARG;
  if (!(eps > 0.0) || !(eps <= 1.0) || !(std::fabs(theta) <= 1e4)) return MG_ERR_ARG;
  if (nu1 < 0 || nu2 < 0 || nu1 > MAX_NU || nu2 > MAX_NU) return MG_ERR_ARG;
  mg_ctx* h = new (std::nothrow) mg_ctx();
  if (!h) return MG_ERR_NOMEM;
  h->n = n; h->k = k; h->levels = levels; h->nu1 = nu1; h->nu2 = nu2; h->eps = eps; h->theta = theta;
  set_geometry(h);
  auto fail = [&](int st) {
    mg_destroy(h);
    return st;
  };
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) return fail(MG_ERR_CUDA);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || h->sms < 1)
      return fail(MG_ERR_CUDA);
  }
  int st = alloc_levels(h);
  if (st < 0) return fail(st);
  const int nc = h->lv[levels - 1].n, N = nc * nc;
  const size_t np = std::max(pass_grid_blocks(n), apply_grid_blocks(n)) + VEC_BLOCKS;
  h->npartial = np;
#define ALLOC(ptr, bytes) \
  if (cudaMalloc(&(ptr), (bytes)) != cudaSuccess) return fail(MG_ERR_NOMEM)
  ALLOC(h->coef, sizeof(double) * MAXL * NCOEF);
  ALLOC(h->coef32, sizeof(float) * MAXL * NCOEF);
  ALLOC(h->stencils, sizeof(double) * MAXL * 9);
  ALLOC(h->dstencil, sizeof(double) * 18);
  ALLOC(h->ltab, sizeof(double) * line_tab_size(k, levels, 1));  // the semi-coarsening layout is the larger
  ALLOC(h->ltab32, sizeof(float) * line_tab_size(k, levels, 1));
  ALLOC(h->linv, sizeof(double) * std::max<size_t>(1, line_inv_offset(k, levels, 0)));
  ALLOC(h->cmap, sizeof(double) * MAP_CLASSES * 2 * MAP_S * MAP_S);
  ALLOC(h->cmap32, sizeof(float) * MAP_CLASSES * 2 * MAP_S * MAP_S);
  ALLOC(h->partial, sizeof(double) * np);
  ALLOC(h->partial2, sizeof(double) * np);
  ALLOC(h->scal, sizeof(double) * NSCAL);
  ALLOC(h->ints, sizeof(int) * NINT);
  if (N > 1) {
    ALLOC(h->cinv, sizeof(double) * N * N);
    ALLOC(h->cinv32, sizeof(float) * N * N);
    ALLOC(h->work, sizeof(double) * N * N);
  }
#undef ALLOC
  if (cudaMemsetAsync(h->ints, 0, sizeof(int) * NINT, h->own) != cudaSuccess) return fail(MG_ERR_CUDA);
  if (cudaMemsetAsync(h->scal, 0, sizeof(double) * NSCAL, h->own) != cudaSuccess) return fail(MG_ERR_CUDA);
  if ((st = run_setup_kernels(h)) < 0) return fail(st);
  if ((st = set_all_smem_attrs<double>()) < 0 || (st = set_all_smem_attrs<float>()) < 0) return fail(st);
  // the cluster support of the fused calls, checked here, outside any stream capture
  call_cluster_supported<double, false>();
  call_cluster_supported<double, true>();
  call_cluster_supported<float, false>();
  call2_cluster_supported<double>();
  call2_cluster_supported<float>();
  h->ok = true;
  *out = h;
  return MG_OK;
}

int mg_set_option(mg_handle h, int key, double value) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  switch (key) {
    case MG_OPT_OMEGA: {
      if (!(value > 0.0) || !(value < 2.0)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->omega = value;
      drop_graphs(h);
      return run_setup_kernels(h);
    }
    case MG_OPT_TMA_PASSES: {
      if (!(value == 0.0 || value == 1.0)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->tma32 = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_CONDENSED_CHILDREN: {
      if (!(value == 0.0 || value == 1.0)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->condense = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_DEEP_CALLS: {
      const int c = (int)value;
      if (value != (double)c || !(c == 0 || c == 63 || c == 127 || c == 255 || c == 511)) return MG_ERR_ARG;
      if (c && h->batched) return MG_ERR_ARG;  // cooperative launches in concurrent graph branches
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->deep_n = c;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_TEST_STALL_BARRIER: {
      if (!(value >= -1.0 && value <= 1e6 && value == (double)(int)value)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->stall_cta = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_TEST_STALL_COPY: {
      if (!(value >= -1.0 && value <= 1e9 && value == (double)(int)value)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->stall_tile = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_COARSE_OP: {
      if (!(value == 0.0 || value == 1.0)) return MG_ERR_ARG;
      if (h->semi && value != 0.0) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->rediscretized = (int)value;
      drop_graphs(h);
      return run_setup_kernels(h);
    }
    case MG_OPT_STOP: {
      if (!(value == 0.0 || value == 1.0)) return MG_ERR_ARG;
      h->stop_rule = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_SMOOTHER: {
      if (!(value == 0.0 || value == 1.0 || value == 2.0)) return MG_ERR_ARG;
      if (h->semi && value != 2.0) return MG_ERR_ARG;
      if (h->nonsym && value != 0.0) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->smoother = (int)value;
      h->maps_ok = h->maps32_ok = false;
      h->pm_ok = h->pm32_ok = false;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_CONV_X:
    case MG_OPT_CONV_Y: {
      if (!(std::fabs(value) <= 1e12)) return MG_ERR_ARG;
      const double bx = key == MG_OPT_CONV_X ? value : h->bx, by = key == MG_OPT_CONV_Y ? value : h->by;
      if ((bx != 0.0 || by != 0.0) && (h->smoother != 0 || h->semi)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      h->bx = bx;
      h->by = by;
      h->nonsym = bx != 0.0 || by != 0.0;
      drop_graphs(h);
      return run_setup_kernels(h);
    }
    case MG_OPT_PRECOND: {
      if (!(value == 0.0 || value == 1.0)) return MG_ERR_ARG;
      h->precond = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_FUSED_CALL: {
      if (!(value == 0.0 || value == 1.0 || value == 2.0)) return MG_ERR_ARG;
      h->fused = (int)value;
      drop_graphs(h);
      return MG_OK;
    }
    case MG_OPT_COARSENING: {
      if (!(value == 0.0 || value == 1.0)) return MG_ERR_ARG;
      if (value == 1.0 && (h->levels != h->k || h->rediscretized || h->nonsym)) return MG_ERR_ARG;
      if ((int)value == h->semi) return MG_OK;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      drop_graphs(h);
      KC_TRY(free_levels(h));
      h->semi = (int)value;
      h->smoother = h->semi ? 2 : 0;
      KC_TRY(alloc_levels(h));
      KC_CUDA(cudaStreamSynchronize(h->own));
      return run_setup_kernels(h);
    }
    case MG_OPT_COARSE_N:
    case MG_OPT_COARSE_N32: {
      const int c = (int)value;
      if (value != (double)c || !(c == 1 || c == 3 || c == 7 || c == 15 || c == 31 || c == 63)) return MG_ERR_ARG;
      KC_CUDA(cudaStreamSynchronize(h->stream()));
      drop_graphs(h);
      KC_TRY(free_levels(h));
      if (key == MG_OPT_COARSE_N) h->coarse_n = c; else h->coarse_n32 = c;
      KC_TRY(alloc_levels(h));
      KC_CUDA(cudaStreamSynchronize(h->own));
      return MG_OK;
    }
    default: return MG_ERR_ARG;
  }
}

int mg_get_option(mg_handle h, int key, double* value) {
  if (!value) return MG_ERR_ARG;
  if (!valid_handle(h)) return MG_ERR_STATE;
  switch (key) {
    case MG_OPT_OMEGA: *value = h->omega; return MG_OK;
    case MG_OPT_COARSE_N: *value = h->coarse_n; return MG_OK;
    case MG_OPT_COARSE_N32: *value = h->coarse_n32; return MG_OK;
    case MG_OPT_COARSE_OP: *value = h->rediscretized; return MG_OK;
    case MG_OPT_STOP: *value = h->stop_rule; return MG_OK;
    case MG_OPT_SMOOTHER: *value = h->smoother; return MG_OK;
    case MG_OPT_COARSENING: *value = h->semi; return MG_OK;
    case MG_OPT_PRECOND: *value = h->precond; return MG_OK;
    case MG_OPT_FUSED_CALL: *value = h->fused; return MG_OK;
    case MG_OPT_TMA_PASSES: *value = h->tma32; return MG_OK;
    case MG_OPT_CONDENSED_CHILDREN: *value = h->condense; return MG_OK;
    case MG_OPT_TEST_STALL_COPY: *value = h->stall_tile; return MG_OK;
    case MG_OPT_TEST_STALL_BARRIER: *value = h->stall_cta; return MG_OK;
    case MG_OPT_DEEP_CALLS: *value = h->deep_n; return MG_OK;
    case MG_OPT_CONV_X: *value = h->bx; return MG_OK;
    case MG_OPT_CONV_Y: *value = h->by; return MG_OK;
    case MG_OPT_LEVELS: *value = h->levels; return MG_OK;
    case MG_OPT_N: *value = h->n; return MG_OK;
    case MG_OPT_LAUNCHES: *value = h->last_launches; return MG_OK;
    default: return MG_ERR_ARG;
  }
}

int mg_set_stream(mg_handle h, void* stream) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  h->ext = (cudaStream_t)stream;
  h->has_ext = stream != nullptr;
  return MG_OK;
}

static int kcycle_common(mg_handle h, double* v, const double* f, int kappa, bool adjoint) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !f || kappa < 1) return MG_ERR_ARG;
  if (adjoint && (h->smoother != 0 || h->nonsym)) return MG_ERR_ARG;
  trim_graphs(h);
  GraphEntry* ge;
  KC_TRY(get_cycle_graph(h, v, f, kappa, adjoint ? 2 : 0, &ge));
  KC_CUDA(cudaGraphLaunch(ge->exec, h->stream()));
  return MG_OK;
}

int mg_kcycle(mg_handle h, double* v, const double* f, int kappa) { return kcycle_common(h, v, f, kappa, false); }

int mg_kcycle_adjoint(mg_handle h, double* v, const double* f, int kappa) {
  return kcycle_common(h, v, f, kappa, true);
}

int mg_solve(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles, int* cycles,
             double* final_relres, double* history) {
  return solve_impl(h, v, f, kappa, tol, max_cycles, cycles, final_relres, history);
}

int mg_solve_adjoint(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles, int* cycles,
                     double* final_relres, double* history) {
  return solve_impl(h, v, f, kappa, tol, max_cycles, cycles, final_relres, history, true);
}

int mg_solve_host(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles, int* cycles,
                  double* final_relres, double* history) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !f) return MG_ERR_ARG;
  const size_t bytes = sizeof(double) * (size_t)h->n * h->n;
  if (!h->hv) KC_CUDA(cudaMalloc(&h->hv, bytes));
  if (!h->hf) KC_CUDA(cudaMalloc(&h->hf, bytes));
  cudaStream_t s = h->stream();
  KC_CUDA(cudaMemcpyAsync(h->hf, f, bytes, cudaMemcpyHostToDevice, s));
  KC_CUDA(cudaMemcpyAsync(h->hv, v, bytes, cudaMemcpyHostToDevice, s));
  const int st = solve_impl(h, h->hv, h->hf, kappa, tol, max_cycles, cycles, final_relres, history);
  if (st < 0) return st;
  KC_CUDA(cudaMemcpyAsync(v, h->hv, bytes, cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  return st;
}

static int pcg_impl(mg_handle h, double* x, const double* b, int kappa, double tol, int max_iters, int flexible,
                    bool mixed, int* iters, double* final_relres, double* history) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!x || !b || kappa < 1 || !(tol > 0) || max_iters < 1) return MG_ERR_ARG;
  const bool sym = h->precond == 1;
  if (sym && (mixed || h->smoother != 0)) return MG_ERR_ARG;  // the adjoint cycle: FP64 damped Jacobi
  if (h->nonsym) return MG_ERR_ARG;                            // CG needs a symmetric operator
  trim_graphs(h);
  const size_t len = (size_t)h->n * h->n, bytes = sizeof(double) * len;
  double** vecs[] = {&h->pr, &h->pp, &h->pq, &h->pz, &h->pzold};
  for (double** p : vecs)
    if (!*p) KC_CUDA(cudaMalloc(p, bytes));
  if (sym) {
    if (!h->pw) KC_CUDA(cudaMalloc(&h->pw, bytes));
    if (!h->pz2) KC_CUDA(cudaMalloc(&h->pz2, bytes));
  }
  if (mixed) KC_TRY(ensure_levels32(h));
  KC_TRY(ensure_hist(h, max_iters));
  cudaStream_t s = h->stream();
  const int* done = h->ints + I_DONE;
  float* r32 = h->lv[0].f32;
  float* z32 = h->lv[0].v32;
  // z = B r from a zero start: FP64 cycle, or r -> FP32, FP32 cycle, z <- FP64; symmetrised:
  // z = B r, w = r - A z, z += B^T w (the adjoint cycle from zero)
  auto emit_precond = [&](cudaStream_t o, const int* skip) -> int {
    if (!mixed) {
      Binding bz{h->pz, h->pr, h->n};
      KC_TRY(emit_cycle(h, bz, kappa, true, false, false, skip, o));
      if (!sym) return MG_OK;
      const int n = h->n;
      dim3 agrid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
      apply_kernel<double, NT_VEC><<<agrid, NT_VEC, 0, o>>>(h->pz, h->pr, h->pw, h->coef, 0, n, n, nullptr, skip);
      KC_CUDA(cudaGetLastError());
      ++h->launch_count;
      Binding bw{h->pz2, h->pw, h->n};
      KC_TRY(emit_cycle(h, bw, kappa, true, true, false, skip, o));
      vec_add_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, o>>>(h->pz, h->pz2, len, skip);
      KC_CUDA(cudaGetLastError());
      ++h->launch_count;
      return MG_OK;
    }
    const int n = h->n;
    dim3 cgrid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
    convert_kernel<NT_VEC, double, float><<<cgrid, NT_VEC, 0, o>>>(r32, h->ld32_0, h->pr, n, n, skip);
    BindingT<float> b32{z32, r32, h->ld32_0};
    KC_TRY(emit_cycle(h, b32, kappa, true, false, false, skip, o));
    convert_kernel<NT_VEC, float, double><<<cgrid, NT_VEC, 0, o>>>(h->pz, n, z32, h->ld32_0, n, skip);
    KC_CUDA(cudaGetLastError());
    h->launch_count += 2;
    return MG_OK;
  };
  const int fl = (flexible ? 1 : 0) | (mixed ? 2 : 0) | (sym ? 4 : 0);
  GraphEntry* ge = find_graph(h, G_PCG, kappa, fl, x, b);
  if (!ge) {
    GraphEntry e;
    e.kind = G_PCG; e.kappa = kappa; e.flag = fl; e.p0 = x; e.p1 = b;
    const int napply = (int)apply_grid_blocks(h->n);
    KC_TRY(build_while_graph(h, [&](cudaGraphConditionalHandle ch) -> int {
      cudaStream_t o = h->own;
      const int n = h->n;
      dim3 grid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
      apply_dot_kernel<NT_VEC><<<grid, NT_VEC, 0, o>>>(h->pp, h->pq, h->coef, n, h->partial, done);
      pcg_alpha_kernel<NT_VEC><<<1, NT_VEC, 0, o>>>(h->partial, napply, h->scal, h->ints);
      pcg_update_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, o>>>(x, h->pr, h->pp, h->pq, len, h->scal, h->partial,
                                                             h->ints);
      finish_step_kernel<NT_VEC><<<1, NT_VEC, 0, o>>>(h->partial, VEC_BLOCKS, h->scal, h->ints, h->hist, ch, 1);
      KC_CUDA(cudaGetLastError());
      KC_TRY(emit_precond(o, done));
      dot_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, o>>>(h->pr, h->pz, (fl & 1) ? h->pzold : nullptr, len, h->partial,
                                                       h->partial2, done);
      pcg_beta_kernel<NT_VEC><<<1, NT_VEC, 0, o>>>(h->partial, h->partial2, VEC_BLOCKS, fl & 1, h->scal, h->ints);
      pcg_p_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, o>>>(h->pp, h->pz, (fl & 1) ? h->pzold : nullptr, len, h->scal, 1,
                                                         h->ints);
      KC_CUDA(cudaGetLastError());
      h->launch_count += 7;
      return MG_OK;
    }, &e.graph, &e.exec));
    e.launches = h->launch_count;
    ge = add_graph(h, e);
  }
  // initialisation: x = 0, r = b, z = B r, p = z, rz = r.z
  KC_CUDA(cudaMemsetAsync(x, 0, bytes, s));
  KC_CUDA(cudaMemcpyAsync(h->pr, b, bytes, cudaMemcpyDeviceToDevice, s));
  KC_TRY(launch_norm2(h, b, h->scal + S_FNORM2, s));
  reset_state_kernel<<<1, 1, 0, s>>>(h->ints, max_iters, h->scal, tol);
  KC_CUDA(cudaGetLastError());
  KC_TRY(emit_precond(s, nullptr));
  pcg_p_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, s>>>(h->pp, h->pz, (fl & 1) ? h->pzold : nullptr, len, h->scal, 0,
                                                     h->ints);
  dot_kernel<NT_VEC><<<VEC_BLOCKS, NT_VEC, 0, s>>>(h->pr, h->pz, nullptr, len, h->partial, nullptr, nullptr);
  sum_to_scalar_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(h->partial, VEC_BLOCKS, h->scal + S_RZ);
  KC_CUDA(cudaGetLastError());
  KC_CUDA(cudaGraphLaunch(ge->exec, s));
  return read_result(h, s, tol, iters, final_relres, history);
}

int mg_pcg(mg_handle h, double* x, const double* b, int kappa, double tol, int max_iters, int flexible, int* iters,
           double* final_relres, double* history) {
  return pcg_impl(h, x, b, kappa, tol, max_iters, flexible, false, iters, final_relres, history);
}

int mg_pcg_mixed(mg_handle h, double* x, const double* b, int kappa, double tol, int max_iters, int flexible,
                 int* iters, double* final_relres, double* history) {
  return pcg_impl(h, x, b, kappa, tol, max_iters, flexible, true, iters, final_relres, history);
}

int mg_kcycle_f32(mg_handle h, float* v, const float* f, int kappa) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !f || kappa < 1) return MG_ERR_ARG;
  trim_graphs(h);
  KC_TRY(ensure_levels32(h));
  GraphEntry* ge = find_graph(h, G_CYCLE32, kappa, 0, v, f);
  if (!ge) {
    BindingT<float> b{v, f, h->n};
    cudaGraph_t g;
    h->launch_count = 0;
    KC_CUDA(cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal));
    const int st = emit_cycle(h, b, kappa, false, false, false, nullptr, h->own);
    const cudaError_t ce = cudaStreamEndCapture(h->own, &g);
    if (st < 0) {
      if (ce == cudaSuccess) cudaGraphDestroy(g);
      return st;
    }
    KC_CUDA(ce);
    GraphEntry e;
    e.kind = G_CYCLE32; e.kappa = kappa; e.p0 = v; e.p1 = f; e.graph = g; e.launches = h->launch_count;
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(g);
      KC_CUDA(ie);
    }
    ge = add_graph(h, e);
  }
  KC_CUDA(cudaGraphLaunch(ge->exec, h->stream()));
  return MG_OK;
}

int mg_solve_mixed(mg_handle h, double* x, const double* f, int kappa, double tol, int max_iters, int* iters,
                   double* final_relres, double* history) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!x || !f || kappa < 1 || !(tol > 0) || max_iters < 1) return MG_ERR_ARG;
  trim_graphs(h);
  KC_TRY(ensure_levels32(h));
  KC_TRY(ensure_hist(h, max_iters));
  cudaStream_t s = h->stream();
  const int n = h->n;
  float* d = h->lv[0].v32;
  float* r32 = h->lv[0].f32;
  const int napply = (int)apply_grid_blocks(n);
  dim3 agrid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
  GraphEntry* ge = find_graph(h, G_MIXED, kappa, 0, x, f);
  if (!ge) {
    GraphEntry e;
    e.kind = G_MIXED; e.kappa = kappa; e.p0 = x; e.p1 = f;
    BindingT<float> b{d, r32, h->ld32_0};
    const int* done = h->ints + I_DONE;
    KC_TRY(build_while_graph(h, [&](cudaGraphConditionalHandle ch) -> int {
      cudaStream_t o = h->own;
      // d = B r (FP32 kappa-cycle from zero), x += d, r = f - A x (FP64), stopping test
      KC_TRY(emit_cycle(h, b, kappa, true, false, false, done, o));
      ir_add_kernel<NT_VEC><<<agrid, NT_VEC, 0, o>>>(x, d, n, h->ld32_0, done);
      ir_residual_kernel<NT_VEC><<<agrid, NT_VEC, 0, o>>>(x, f, r32, h->ld32_0, h->coef, n, h->partial, done);
      finish_step_kernel<NT_VEC><<<1, NT_VEC, 0, o>>>(h->partial, napply, h->scal, h->ints, h->hist, ch, 1);
      KC_CUDA(cudaGetLastError());
      h->launch_count += 3;
      return MG_OK;
    }, &e.graph, &e.exec));
    e.launches = h->launch_count;
    ge = add_graph(h, e);
  }
  KC_TRY(launch_norm2(h, f, h->scal + S_FNORM2, s));
  reset_state_kernel<<<1, 1, 0, s>>>(h->ints, max_iters, h->scal, tol);
  ir_residual_kernel<NT_VEC><<<agrid, NT_VEC, 0, s>>>(x, f, r32, h->ld32_0, h->coef, n, h->partial, nullptr);
  KC_CUDA(cudaGetLastError());
  KC_CUDA(cudaGraphLaunch(ge->exec, s));
  return read_result(h, s, tol, iters, final_relres, history);
}

int mg_apply(mg_handle h, const double* v, double* out) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !out) return MG_ERR_ARG;
  return emit_apply(h, v, nullptr, out, nullptr, nullptr, h->stream());
}

int mg_residual_norm(mg_handle h, const double* v, const double* f, double* norm) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !f || !norm) return MG_ERR_ARG;
  cudaStream_t s = h->stream();
  KC_TRY(emit_apply(h, v, f, nullptr, h->partial, nullptr, s));
  sum_to_scalar_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(h->partial, (int)apply_grid_blocks(h->n), h->scal + S_LAST);
  KC_CUDA(cudaGetLastError());
  double r2;
  KC_CUDA(cudaMemcpyAsync(&r2, h->scal + S_LAST, sizeof(double), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  *norm = std::sqrt(r2);
  return MG_OK;
}

int mg_param_grads(mg_handle h, const double* lambda, const double* u, double* dtheta, double* deps) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!lambda || !u || !dtheta || !deps) return MG_ERR_ARG;
  cudaStream_t s = h->stream();
  const int n = h->n;
  dim3 grid((n + 31) / 32, (n + NT_VEC / 32 - 1) / (NT_VEC / 32));
  grad_kernel<NT_VEC><<<grid, NT_VEC, 0, s>>>(lambda, u, n, h->dstencil, h->partial, h->partial2);
  const int np = (int)apply_grid_blocks(n);
  sum_to_scalar_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(h->partial, np, h->scal + S_ALPHA);
  sum_to_scalar_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(h->partial2, np, h->scal + S_BETA);
  KC_CUDA(cudaGetLastError());
  double r[NSCAL];
  KC_CUDA(cudaMemcpyAsync(r, h->scal, sizeof(r), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  *dtheta = -r[S_ALPHA];
  *deps = -r[S_BETA];
  return MG_OK;
}

int mg_stencils(mg_handle h, double* out, int max_levels, int* written) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!out || max_levels < 1) return MG_ERR_ARG;
  const int nl = std::min(max_levels, h->levels);
  KC_CUDA(cudaStreamSynchronize(h->stream()));
  KC_CUDA(cudaMemcpy(out, h->stencils, sizeof(double) * 9 * nl, cudaMemcpyDeviceToHost));
  if (written) *written = nl;
  return MG_OK;
}

int mg_counters(mg_handle h, int kappa, long long* calls_per_level, long long* launches, long long* coarse_calls) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (kappa < 1) return MG_ERR_ARG;
  ensure_maps(h);  // whether calls run condensed or fused depends on the maps being available
  // walk Algorithm 3's recursion, counting only
  std::vector<long long> calls(h->levels, 0);
  long long fine_launches = 0, coarse = 0, absorbed = 0;
  struct Walk {
    mg_ctx* h;
    std::vector<long long>& calls;
    long long& fine_launches;
    long long& coarse;
    long long& absorbed;  // calls just above the coarse kernel's that run inside a larger launch
    void call(int l, int kap, bool inside = false, bool deep = false) {
      calls[l] += 1;
      if (l >= h->lc) ++coarse;
      if (l == h->levels - 1) {
        if (h->semi) ++fine_launches;  // the one-row line solve
        return;
      }
      if (deep && l < h->lc) {  // inside a persistent deep launch, with its condensed child calls
        if (l + 1 == h->lc) ++absorbed;
        call(l + 1, kap, false, true);
        if (kap > 1) call(l + 1, kap - 1, false, true);
        return;
      }
      if (inside) {  // part of its parent's two-level launch
        ++absorbed;
        call(l + 1, kap);
        if (kap > 1) call(l + 1, kap - 1);
        return;
      }
      if (l < h->lc && deep_ok<double>(h, l, false)) {
        ++fine_launches;  // one launch for the call and everything below it
        if (l + 1 == h->lc) ++absorbed;
        call(l + 1, kap, false, true);
        if (kap > 1) call(l + 1, kap - 1, false, true);
        return;
      }
      if (l < h->lc && fused2_ok<double>(h, l, kap, false)) {
        ++fine_launches;  // one launch for the call and its child calls
        call(l + 1, kap, true);
        if (kap > 1) call(l + 1, kap - 1, true);
        return;
      }
      if (l < h->lc) {
        if (fused_call_ok<double>(h, l, false)) {
          // one cluster launch: counted with the coarse-kernel launches below
        } else if (h->smoother == 0) {
          fine_launches += 2;  // pass A + pass B
        } else {                // line launches (two per relaxation), restriction, folded prolongation
          fine_launches += (h->nu1 > 0 ? 2 * h->nu1 : 0) + 1 + (h->nu2 > 0 ? 2 * h->nu2 : 1);
        }
      }
      call(l + 1, kap);
      if (kap > 1) call(l + 1, kap - 1);
    }
  } w{h, calls, fine_launches, coarse, absorbed};
  w.call(0, std::min(kappa, h->levels + 1));
  // one coarse-kernel launch serves both calls of a fine parent (or the whole cycle when lc == 0)
  const long long coarse_launches = h->lc >= h->levels ? 0 : (h->lc == 0 ? 1 : calls[h->lc - 1] - absorbed);
  if (calls_per_level)
    for (int l = 0; l < h->levels; ++l) calls_per_level[l] = calls[l];
  if (launches) *launches = fine_launches + coarse_launches;
  if (coarse_calls) *coarse_calls = coarse;
  return MG_OK;
}

int mg_level_grid(mg_handle h, int level, int fp32, int* n_level, int* ctas) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!n_level || !ctas || level < 0 || level >= h->levels) return MG_ERR_ARG;
  if (h->smoother != 0 || h->semi) return MG_ERR_ARG;
  ensure_maps(h);  // deep and condensed calls depend on the maps being available
  const int n = h->lv[level].n;
  *n_level = n;
  int lc = h->lc;
  if (fp32) {  // the FP32 coarse level, as ensure_levels32 places it
    lc = h->levels - 1;
    for (int l = 0; l < h->levels; ++l)
      if (h->lv[l].n <= h->coarse_n32) {
        lc = l;
        break;
      }
  }
  if (level >= lc) {
    *ctas = 1;
    return MG_OK;
  }
  for (int l = 1; l <= level; ++l)
    if (fp32 ? deep_ok<float>(h, l, false) : deep_ok<double>(h, l, false)) {
      DeepShape sh;  // inside a persistent deep launch
      if (fp32 ? deep_shape<float>(h, l, &sh) : deep_shape<double>(h, l, &sh)) *ctas = sh.grid;
      return MG_OK;
    }
  if (h->fused >= 2 && h->condense && !h->nonsym && level >= 1 && level + 2 == lc && h->lv[lc].n <= PM_MAX_SIDE &&
      (fp32 ? call2_cluster_supported<float>() : call2_cluster_supported<double>())) {
    *ctas = CALL_MAX_CTAS;  // the call runs with its child calls as one cluster launch
    return MG_OK;
  }
  if (fp32 ? fused_call_ok<float>(h, level, false, lc) : fused_call_ok<double>(h, level, false, lc)) {
    *ctas = fp32 ? call_ctas<float>(h, level) : call_ctas<double>(h, level);
    return MG_OK;
  }
  if (fp32 && h->tma32 && n >= TMA_MIN_N && h->nu1 == 2 && h->nu2 == 2 && tensor_map_encoder()) {
    // the persistent tensor-copy passes (pass B's shape shown): every resident slot, at most one per tile
    const int kind = tma_kind(TMA_B, n), ty = tma_ty(kind), tiles = ((n + TM_TX - 1) / TM_TX) * ((n + ty - 1) / ty);
    *ctas = kind == TMA_B ? tma_grid(h, pass_b_tma32<TMA_TY_B>, kind, tiles) : tma_grid(h, pass_b_tma32<TMA_TY_S>, kind, tiles);
    return MG_OK;
  }
  if (fp32 && n >= F32_FAST_MIN && std::max(h->nu1, h->nu2) <= 2) {  // the fast-eligible levels (fast32_ok)
    if (f32_tile_pass_b(n)) {  // (pass A always runs as tiles; pass B's shape shown)
      *ctas = ((n + T32_TX - 1) / T32_TX) * ((n + T32_TY - 1) / T32_TY);
    } else {
      const int strips = (n + SF_COLS - 1) / SF_COLS, R = stream_rows(n);
      *ctas = ((strips + SF_WARPS - 1) / SF_WARPS) * ((n + R - 1) / R);
    }
    return MG_OK;
  }
  const int w = (!fp32 && level >= 1 && !h->nonsym && !h->batched) ? wide_edge(n, h->sms) : 0;
  const int bx = w ? w : tile_edge(n), by = w ? w : tile_rows(n, false);
  *ctas = ((n + bx - 1) / bx) * ((n + by - 1) / by);
  return MG_OK;
}

int mg_profile_cycle(mg_handle h, double* v, const double* f, int kappa, int with_norm, int max_records,
                     double* ms, int* kind, int* level, int* count) {
  if (!valid_handle(h)) return MG_ERR_STATE;
  if (!v || !f || kappa < 1 || max_records < 0) return MG_ERR_ARG;
  cudaStream_t s = h->stream();
  Binding b{v, f, h->n};
  const bool fp32 = (with_norm & 2) != 0;
  if (fp32) KC_TRY(ensure_levels32(h));
  ensure_maps(h);  // the same condensed calls as the graphs of a cycle or a solve
  h->pev.clear();
  h->pkind.clear();
  h->plevel.clear();
  h->prof = true;
  // bit 2: the launches and their event pairs captured into a graph and replayed once, as a
  // solve's graph runs them (no host launch latency inside a pair)
  const bool in_graph = (with_norm & 4) != 0;
  h->prof_graph = in_graph;
  cudaStream_t es = in_graph ? h->own : s;
  if (in_graph) {
    KC_CUDA(cudaStreamSynchronize(s));
    KC_CUDA(cudaStreamBeginCapture(es, cudaStreamCaptureModeThreadLocal));
  }
  int st;
  if (fp32) {  // the FP32 cycle of the mixed path: d = B32 r from zero on the handle's FP32 arrays
    BindingT<float> b32{h->lv[0].v32, h->lv[0].f32, h->ld32_0};
    st = emit_cycle(h, b32, kappa, true, false, false, nullptr, es);
  } else if ((with_norm & 1) && prenorm_ok(h)) {  // the launches of a stand-alone solve cycle
    st = emit_solve_cycle_prenorm(h, b, kappa, cudaGraphConditionalHandle{}, nullptr, es, false);
  } else {
    st = emit_cycle(h, b, kappa, false, false, (with_norm & 1) != 0, nullptr, es);
  }
  h->prof = false;
  h->prof_graph = false;
  if (in_graph) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(es, &g);
    if (st >= 0 && ce != cudaSuccess) st = MG_ERR_CUDA;
    if (st >= 0 && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = MG_ERR_CUDA;
    if (st >= 0 && cudaGraphLaunch(ge, s) != cudaSuccess) st = MG_ERR_CUDA;
    if (st >= 0 && cudaStreamSynchronize(s) != cudaSuccess) st = MG_ERR_CUDA;
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (st == MG_ERR_CUDA) snprintf(g_err, sizeof(g_err), "mg_profile_cycle: graph replay failed");
    cudaGetLastError();
  }
  int result = st;
  if (st >= 0) {
    const cudaError_t se = cudaStreamSynchronize(s);
    if (se != cudaSuccess) {
      snprintf(g_err, sizeof(g_err), "mg_profile_cycle: %s", cudaGetErrorString(se));
      result = MG_ERR_CUDA;
    }
  }
  const int nrec = (int)h->pkind.size();
  if (result >= 0) {
    for (int r = 0; r < nrec && r < max_records; ++r) {
      float t = 0.f;
      cudaEventElapsedTime(&t, h->pev[2 * r], h->pev[2 * r + 1]);
      if (ms) ms[r] = t;
      if (kind) kind[r] = h->pkind[r];
      if (level) level[r] = h->plevel[r];
    }
    if (count) *count = nrec;
  }
  for (cudaEvent_t e : h->pev) cudaEventDestroy(e);
  h->pev.clear();
  return result;
}

int mg_fp64_rate(double* ops_per_second) {
  if (!ops_per_second) return MG_ERR_ARG;
  int dev = 0, sms = 0;
  KC_CUDA(cudaGetDevice(&dev));
  KC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  KC_CUDA(cudaMalloc(&sink, sizeof(double)));
  cudaEvent_t e0, e1;
  KC_CUDA(cudaEventCreate(&e0));
  KC_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * 8, threads = 256, iters = 4000;
  fp64_rate_kernel<<<blocks, threads>>>(sink, 10, 0.999, 1e-3);  // warm-up
  KC_CUDA(cudaEventRecord(e0));
  fp64_rate_kernel<<<blocks, threads>>>(sink, iters, 0.999, 1e-3);
  KC_CUDA(cudaEventRecord(e1));
  KC_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  KC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *ops_per_second = (double)blocks * threads * iters * 8 / (ms * 1e-3);
  return MG_OK;
}

}  // extern "C"

// ============================================================================================
// Batched solves: many independent instances (ragged sizes, own theta and eps) in one graph
// launch, one branch per instance.
// ============================================================================================
struct mg_batch_ctx {
  std::vector<mg_handle> inst;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;  // pointers, kappa, tol, max_iters, mixed of the cached graph
};

namespace {
void batch_drop_graph(mg_batch_ctx* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key.clear();
}

// Time `reps` kappa-cycles of handle h in the given precision (ms per cycle) on scratch arrays.
// The autotuner's launch shape of one instance.
struct TuneShape {
  int thr, fused, condensed, tma;
};
constexpr size_t TUNE_MAX_INSTANCES = 64;  // instances of one side timed together (the memory pressure of the batch)
constexpr int TUNE_ITERS = 4;             // solve iterations timed per candidate

// ms per iteration of the instances `hs` solved together, as in a batch: one graph holding each
// instance's solve branch (initialisation, then TUNE_ITERS iterations; a tolerance of 1e-300 keeps
// every branch running), launched once to warm up and once timed.
int time_subbatch(const std::vector<mg_handle>& hs, cudaStream_t s, int kappa, bool mixed, int iters,
                  const std::vector<double*>& xs, const std::vector<double*>& fs, float* ms_out) {
  for (mg_handle h : hs) {
    KC_TRY(ensure_hist(h, iters));
    if (mixed) KC_TRY(ensure_levels32(h));
    trim_graphs(h);  // builds the maps the options call for
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  KC_CUDA(cudaGraphCreate(&g, 0));
  int st = MG_OK;
  for (size_t i = 0; i < hs.size() && st == MG_OK; ++i)
    st = add_solve_branch(hs[i], g, xs[i], fs[i], kappa, 1e-300, iters, mixed);
  if (st == MG_OK && cudaGraphInstantiate(&e, g, 0) != cudaSuccess) st = MG_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  if (st == MG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = MG_ERR_CUDA;
  if (st == MG_OK && cudaGraphLaunch(e, s) != cudaSuccess) st = MG_ERR_CUDA;  // warm-up
  // the fastest of three timed launches: the shapes' differences are a few percent, about the
  // spread of single launches
  for (int rep = 0; rep < 3 && st == MG_OK; ++rep) {
    float t = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(e, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      st = MG_ERR_CUDA;
    else if (rep == 0 || t < ms)
      ms = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e) cudaGraphExecDestroy(e);
  if (g) cudaGraphDestroy(g);
  if (st != MG_OK) {
    cudaGetLastError();
    return st;
  }
  *ms_out = ms / iters;
  return MG_OK;
}
}  // namespace

extern "C" {

int mg_batch_destroy(mg_batch b) {
  if (!b) return MG_OK;
  batch_drop_graph(b);
  for (mg_handle h : b->inst) mg_destroy(h);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return MG_OK;
}

int mg_batch_create(int count, const int* n, const double* eps, const double* theta, const int* levels, int nu1,
                    int nu2, mg_batch* out) {
  if (!out || count < 1 || !n || !eps || !theta) return MG_ERR_ARG;
  *out = nullptr;
  mg_batch_ctx* b = new (std::nothrow) mg_batch_ctx();
  if (!b) return MG_ERR_NOMEM;
  for (int i = 0; i < count; ++i) {
    int k = 0;
    while (k < 15 && ((1 << k) - 1) < n[i]) ++k;
    mg_handle h = nullptr;
    const int st = mg_setup(n[i], eps[i], theta[i], levels ? levels[i] : k, nu1, nu2, &h);
    if (st < 0) {
      mg_batch_destroy(b);
      return st;
    }
    // no fused calls in a batch: a call cluster holds 16 SMs while one of them walks the coarse
    // levels, SMs the other instances' concurrent branches would use (measured: 256-instance mixed
    // batch 4.2 s without, 4.7 s with)
    h->fused = 0;
    h->batched = true;
    h->deep_n = 0;  // cooperative launches do not go in concurrent graph branches
    b->inst.push_back(h);
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    mg_batch_destroy(b);
    return MG_ERR_CUDA;
  }
  *out = b;
  return MG_OK;
}

int mg_batch_autotune(mg_batch b, int kappa, int mixed, int* chosen) {
  if (!b || kappa < 1) return MG_ERR_ARG;
  // distinct grid sides, largest first (the large instances set the batch's critical path)
  std::vector<int> sizes;
  for (mg_handle h : b->inst)
    if (std::find(sizes.begin(), sizes.end(), h->n) == sizes.end()) sizes.push_back(h->n);
  std::sort(sizes.begin(), sizes.end(), std::greater<int>());
  const int thr_key = mixed ? MG_OPT_COARSE_N32 : MG_OPT_COARSE_N;
  const std::vector<int> cand_thr = mixed ? std::vector<int>{15, 31, 63} : std::vector<int>{7, 15, 31};
  int pos = 0;
  for (int n : sizes) {
    std::vector<mg_handle> all, sub;
    for (mg_handle h : b->inst)
      if (h->n == n) all.push_back(h);
    for (size_t i = 0; i < all.size() && sub.size() < TUNE_MAX_INSTANCES; ++i) sub.push_back(all[i]);
    const size_t len = (size_t)n * n;
    std::vector<double*> xs(sub.size(), nullptr), fs(sub.size(), nullptr);
    int st = MG_OK;
    for (size_t i = 0; i < sub.size() && st == MG_OK; ++i) {
      if (cudaMalloc(&xs[i], len * 8) != cudaSuccess || cudaMalloc(&fs[i], len * 8) != cudaSuccess) st = MG_ERR_NOMEM;
      else if (cudaMemset(fs[i], 0x3f, len * 8) != cudaSuccess) st = MG_ERR_CUDA;  // a positive constant
    }
    auto apply = [&](const std::vector<mg_handle>& hs, const TuneShape& t) -> int {
      for (mg_handle h : hs) {
        KC_TRY(mg_set_option(h, thr_key, t.thr));
        KC_TRY(mg_set_option(h, MG_OPT_FUSED_CALL, t.fused));
        KC_TRY(mg_set_option(h, MG_OPT_CONDENSED_CHILDREN, t.condensed));
        KC_TRY(mg_set_option(h, MG_OPT_TMA_PASSES, t.tma));
      }
      return MG_OK;
    };
    auto measure = [&](const TuneShape& t, float* ms) -> int {
      KC_TRY(apply(sub, t));
      return time_subbatch(sub, b->stream, kappa, mixed != 0, TUNE_ITERS, xs, fs, ms);
    };
    TuneShape best{thr_key == MG_OPT_COARSE_N ? sub[0]->coarse_n : sub[0]->coarse_n32, sub[0]->fused,
                   sub[0]->condense, sub[0]->tma32};
    float best_ms = 1e30f;
    // coordinate descent: the threshold, then fused call x condensed children, then the FP32
    // large-level passes (sides >= 1023 only)
    if (st == MG_OK) {
      for (int c : cand_thr) {
        TuneShape t = best;
        t.thr = c;
        float ms;
        if (measure(t, &ms) == MG_OK && ms < best_ms) { best_ms = ms; best.thr = c; }
      }
      const TuneShape base = best;
      for (int fc = 0; fc < 6; ++fc) {
        TuneShape t = base;
        t.fused = fc % 3;
        t.condensed = fc / 3;
        if (t.fused == base.fused && t.condensed == base.condensed) continue;
        float ms;
        if (measure(t, &ms) == MG_OK && ms < best_ms) { best_ms = ms; best = t; }
      }
      if (mixed && n >= F32_FAST_MIN) {
        TuneShape t = best;
        t.tma = 1 - best.tma;
        float ms;
        if (measure(t, &ms) == MG_OK && ms < best_ms) { best_ms = ms; best = t; }
      }
    }
    for (size_t i = 0; i < sub.size(); ++i) {
      if (xs[i]) cudaFree(xs[i]);
      if (fs[i]) cudaFree(fs[i]);
    }
    cudaGetLastError();
    if (st < 0) return st;
    if (best_ms >= 1e30f) return MG_ERR_CUDA;
    KC_TRY(apply(all, best));
    if (chosen) { chosen[2 * pos] = n; chosen[2 * pos + 1] = best.thr; }
    ++pos;
  }
  batch_drop_graph(b);
  return MG_OK;
}

int mg_batch_instance(mg_batch b, int index, mg_handle* out) {
  if (!b || !out || index < 0 || index >= (int)b->inst.size()) return MG_ERR_ARG;
  *out = b->inst[index];
  return MG_OK;
}

int mg_batch_set_option(mg_batch b, int key, double value) {
  if (!b) return MG_ERR_ARG;
  if (key == MG_OPT_LEVELS || key == MG_OPT_N || key == MG_OPT_LAUNCHES) return MG_ERR_ARG;
  for (mg_handle h : b->inst) KC_TRY(mg_set_option(h, key, value));
  batch_drop_graph(b);
  return MG_OK;
}

int mg_setup_batched(int count, const int* n, const double* eps, const double* theta, int nu1, int nu2,
                     mg_batch* out) {
  return mg_batch_create(count, n, eps, theta, nullptr, nu1, nu2, out);
}

int mg_solve_batched(mg_batch b, double* const* v, const double* const* f, int kappa, double tol, int* cycles) {
  return mg_batch_solve(b, v, f, kappa, tol, 10000, 0, cycles, nullptr);
}

int mg_batch_solve(mg_batch b, double* const* x, const double* const* f, int kappa, double tol, int max_iters,
                   int mixed, int* iters, double* relres) {
  if (!b || !x || !f || kappa < 1 || !(tol > 0) || max_iters < 1) return MG_ERR_ARG;
  const size_t cnt = b->inst.size();
  std::vector<const void*> key;
  for (size_t i = 0; i < cnt; ++i) {
    if (!x[i] || !f[i]) return MG_ERR_ARG;
    key.push_back(x[i]);
    key.push_back(f[i]);
  }
  key.push_back((const void*)(intptr_t)kappa);
  key.push_back((const void*)(intptr_t)max_iters);
  key.push_back((const void*)(intptr_t)mixed);
  double tl = tol;
  const void* tk;
  memcpy(&tk, &tl, sizeof(tk));
  key.push_back(tk);
  if (!b->exec || key != b->key) {
    batch_drop_graph(b);
    for (mg_handle h : b->inst) {
      KC_TRY(ensure_hist(h, max_iters));
      if (mixed) KC_TRY(ensure_levels32(h));
      ensure_maps(h);
    }
    KC_CUDA(cudaGraphCreate(&b->graph, 0));
    for (size_t i = 0; i < cnt; ++i) {
      const int st = add_solve_branch(b->inst[i], b->graph, x[i], f[i], kappa, tol, max_iters, mixed != 0);
      if (st < 0) {
        batch_drop_graph(b);
        return st;
      }
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (ie != cudaSuccess) {
      batch_drop_graph(b);
      KC_CUDA(ie);
    }
    b->key = key;
  }
  KC_CUDA(cudaGraphLaunch(b->exec, b->stream));
  KC_CUDA(cudaStreamSynchronize(b->stream));
  int worst = MG_OK;
  for (size_t i = 0; i < cnt; ++i) {
    mg_handle h = b->inst[i];
    int ints[NINT];
    double scal[NSCAL];
    KC_CUDA(cudaMemcpy(ints, h->ints, sizeof(ints), cudaMemcpyDeviceToHost));
    KC_CUDA(cudaMemcpy(scal, h->scal, sizeof(scal), cudaMemcpyDeviceToHost));
    if (iters) iters[i] = ints[I_COUNT];
    if (relres) relres[i] = scal[S_LAST];
    if (!(scal[S_LAST] <= tol)) worst = MG_NOT_CONVERGED;
  }
  return worst;
}

int mg_batch_size(mg_batch b, int* count) {
  if (!b || !count) return MG_ERR_ARG;
  *count = (int)b->inst.size();
  return MG_OK;
}

}  // extern "C"

// ============================================================================================
// ||f - A v|| without allocating: the whole-grid residual-norm kernel, variant whose scratch
// (stencil coefficients, per-block partial sums, result) lives in one static device array.
// ============================================================================================
namespace {
constexpr int NA_MAX_N = 16383;     // largest grid side accepted
constexpr int NA_BLOCKS = 148 * 4;  // fixed grid of the partial-sum kernel: one partial per block
constexpr int NA_OFF_COEF = 0, NA_OFF_COEF32 = 32, NA_OFF_ST = 48, NA_OFF_DST = 64, NA_OFF_RESULT = 96,
              NA_OFF_PART = 128;
constexpr int NA_DOUBLES = NA_OFF_PART + NA_BLOCKS;  // 720 doubles = 5760 bytes
constexpr int NA_MAX_DEVICES = 64;
}  // namespace

// Every GPU that loads this library holds this array until the process exits. In host code its
// name is only a host-side stand-in; kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

namespace {
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {};

template <int NT>
__global__ void __launch_bounds__(NT) residual_partials_fixed_grid_kernel(const double* __restrict__ v,
                                                                          const double* __restrict__ f, int n,
                                                                          const double* coef, double* partial) {
  __shared__ double red[NT / 32];
  const Coef<double> c = load_coef(coef, 0);
  const size_t len = (size_t)n * n;
  double ss = 0.0;
  for (size_t k = blockIdx.x * (size_t)NT + threadIdx.x; k < len; k += (size_t)gridDim.x * NT) {
    const int j = (int)(k / (size_t)n), i = (int)(k - (size_t)j * n);
    const double r = residual_at(neighbours_global(v, i, j, n, n), f[k], c);
    ss = fma(r, r, ss);
  }
  const double t = block_sum<NT>(ss, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;  // every block writes its slot on every call
}

// Device address of the static scratch on the current device, looked up once per device.
int noalloc_scratch(double** out) {
  int dev = -1;
  KC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) {
    snprintf(g_err, sizeof(g_err), "mg_residual_norm_noalloc: device %d out of range", dev);
    return MG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(g_err, sizeof(g_err), "mg_residual_norm_noalloc: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return MG_OK;
}
}  // namespace

extern "C" int mg_residual_norm_noalloc(int n, double eps, double theta, const double* v, const double* f,
                                        void* cuda_stream, double* norm) {
  if (!v || !f || !norm) {
    snprintf(g_err, sizeof(g_err), "mg_residual_norm_noalloc: v, f and norm must not be NULL");
    return MG_ERR_ARG;
  }
  int k = 0;
  while (k < 15 && ((1 << k) - 1) < n) ++k;
  if (n < 1 || ((1 << k) - 1) != n) {
    snprintf(g_err, sizeof(g_err), "mg_residual_norm_noalloc: n=%d is not 2^k - 1", n);
    return MG_ERR_ARG;
  }
  if (n > NA_MAX_N) {
    snprintf(g_err, sizeof(g_err), "mg_residual_norm_noalloc: n=%d exceeds the maximum grid side %d", n, NA_MAX_N);
    return MG_ERR_ARG;
  }
  if (!(eps > 0.0) || !(eps <= 1.0) || !(std::fabs(theta) <= 1e4)) {
    snprintf(g_err, sizeof(g_err), "mg_residual_norm_noalloc: need 0 < eps <= 1 and |theta| <= 1e4 (eps=%g, theta=%g)",
             eps, theta);
    return MG_ERR_ARG;
  }
  double* sc = nullptr;
  KC_TRY(noalloc_scratch(&sc));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the fine-level stencil of (n, eps, theta) into the scratch (the same setup kernel as mg_setup)
  setup_stencils_kernel<<<1, 32, 0, s>>>(theta, eps, n, 1, 0.8, sc + NA_OFF_COEF,
                                         reinterpret_cast<float*>(sc + NA_OFF_COEF32), sc + NA_OFF_ST,
                                         sc + NA_OFF_DST, 0);
  residual_partials_fixed_grid_kernel<NT_VEC><<<NA_BLOCKS, NT_VEC, 0, s>>>(v, f, n, sc + NA_OFF_COEF,
                                                                          sc + NA_OFF_PART);
  sum_to_scalar_kernel<NT_VEC><<<1, NT_VEC, 0, s>>>(sc + NA_OFF_PART, NA_BLOCKS, sc + NA_OFF_RESULT);
  KC_CUDA(cudaGetLastError());
  double r2 = 0.0;
  KC_CUDA(cudaMemcpyAsync(&r2, sc + NA_OFF_RESULT, sizeof(double), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  *norm = std::sqrt(r2);
  return MG_OK;
}
