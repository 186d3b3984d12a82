// FP32 fused level passes fed by the Tensor Memory Accelerator (TMA), for the large levels of the
// FP32 cycle of the mixed forms (Algorithm 3, steps 2-4 and 7-8, in FP32).
//
// Design (sm_103a). Each pass is a persistent kernel: one CTA per SM walks a list of tiles. A tile
// is 120 output columns x TY output rows; its input window (the tile plus a halo of 4 columns and
// nu+2 / nu rows per side) is brought into shared memory by 2-D tensor copies
// (cp.async.bulk.tensor.2d, completion on an mbarrier), double-buffered: while the CTA computes one
// tile, the copies of its next tile are in flight, so HBM streams continuously and no thread spends
// instructions on addresses, bounds or loads of the inputs. The tensor maps' extents are the grid
// side n, so every point outside [0, n)^2 arrives as zero: the Dirichlet boundary costs nothing.
//
// A stage (a Jacobi sweep, the residual) is computed row by row, one warp per band of rows: lane q
// owns the four staged columns 4q..4q+3 (128 columns per warp, one float4 shared-memory access per
// row), keeps the rows above and below in registers and takes its left and right neighbours from
// the adjacent lanes by warp shuffles. The staged columns 0 and 127 lack one neighbour, so every
// stage corrupts one more column at each side; the 4-column halo covers the three stages plus full
// weighting of pass A, and lanes 1..30 own the 120 output columns. From a zero start the first sweep
// is v1 = w f, formed in registers as the second sweep reads its rows, so that pass has two stages.
// Full weighting is split: the residual stage stores the horizontal sums r(x-1) + 2 r(x) + r(x+1) at
// the odd columns, the last phase combines three rows of them per coarse point.
//
// Outputs (the relaxed v, the coarse right-hand side, pass B's corrected and relaxed v) are written
// from registers with coalesced vector stores.
//
// Waits are bounded: a copy that has not completed after TMA_WAIT_NS nanoseconds of the global timer
// (or TMA_WAIT_LIMIT polls, whichever comes first) sets *err, the CTA waits (bounded again) for the
// copies it has issued and returns; the host reports MG_ERR_TIMEOUT.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include <type_traits>

#include "stream_f32.cuh"

namespace kc {

constexpr int TM_TX = 120;        // output columns per tile
constexpr int TM_P = 128;         // staged columns (TM_TX + 2 * 4)
constexpr int TM_HX = 4;          // staged halo columns per side
constexpr int TM_NT = 256;        // threads per CTA (8 warps); two or three CTAs per SM
constexpr int TM_CP = 72;         // staged coarse columns of pass B (x start rounded down to 4)
constexpr uint64_t TMA_WAIT_NS = 500000000ull;  // a copy gets half a second (it takes microseconds)
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 21;    // and at most this many polls (a poll lasts ~4 us)
constexpr int TM_ERR_TIMEOUT = 1;

// Rows of the staged window of a pass with TY output rows: pass A (nu sweeps, residual, full
// weighting) needs nu + 2 halo rows per side, pass B (correction, nu sweeps) nu.
__host__ __device__ constexpr int tm_rows_a(int ty, int nu) { return ty + 2 * (nu + 2); }
__host__ __device__ constexpr int tm_rows_b(int ty, int nu) { return ty + 2 * nu; }
__host__ __device__ constexpr int tm_crows_b(int ty, int nu) { return (ty + 2 * nu) / 2 + 3; }
__host__ __device__ constexpr size_t tm_align(size_t b) { return (b + 1023) / 1024 * 1024; }

// Shared memory of pass A: per buffer set the window of f (and of v when it does not start from
// zero), double-buffered; one work field; the horizontal full-weighting sums (2 floats per lane and
// row); two mbarriers.
__host__ __device__ constexpr size_t tm_field_a(int ty, int nu) { return tm_align(size_t(TM_P) * tm_rows_a(ty, nu) * 4); }
__host__ __device__ constexpr size_t tm_smem_a(int ty, int nu, bool zero) {
  return (zero ? 2 : 4) * tm_field_a(ty, nu) + tm_field_a(ty, nu) + tm_align(size_t(64) * tm_rows_a(ty, nu) * 4) + 1024;
}
__host__ __device__ constexpr size_t tm_field_b(int ty, int nu) { return tm_align(size_t(TM_P) * tm_rows_b(ty, nu) * 4); }
__host__ __device__ constexpr size_t tm_cfield_b(int ty, int nu) { return tm_align(size_t(TM_CP) * tm_crows_b(ty, nu) * 4); }
__host__ __device__ constexpr size_t tm_smem_b(int ty, int nu) {
  return 2 * (2 * tm_field_b(ty, nu) + tm_cfield_b(ty, nu)) + tm_field_b(ty, nu) + 1024;
}

// ------------------------------------------------------------------------------------------------
// PTX wrappers: mbarrier and 2-D tensor copies (global -> shared, this CTA only)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// The dynamic shared memory rounded up to a 1024-byte boundary (the launch requests 1024 bytes
// more than the layout needs); tensor-copy destinations start on such boundaries.
__device__ __forceinline__ unsigned char* tm_base(unsigned char* p) {
  return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One poll: the thread is suspended until the phase completes or about TMA_POLL_NS nanoseconds
// pass, so a waiting warp takes no issue slots from the other CTAs on its SM.
constexpr uint32_t TMA_POLL_NS = 1000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(TMA_POLL_NS)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < TMA_WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > TMA_WAIT_NS) break;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------------------------------------------
// Row walks over a staged window (row pitch TM_P floats)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ Row6 tm_row(const float* __restrict__ s, int r) {
  const float4 q = *reinterpret_cast<const float4*>(s + r * TM_P + 4 * (threadIdx.x & 31));
  const float v[4] = {q.x, q.y, q.z, q.w};
  return with_halo(v);
}
__device__ __forceinline__ void tm_f4(const float* __restrict__ s, int r, float (&o)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(s + r * TM_P + 4 * (threadIdx.x & 31));
  o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
}
__device__ __forceinline__ void tm_st4(float* __restrict__ s, int r, const float (&o)[4]) {
  *reinterpret_cast<float4*>(s + r * TM_P + 4 * (threadIdx.x & 31)) = make_float4(o[0], o[1], o[2], o[3]);
}

// Rows [R0, R0 + NROWS) split into contiguous bands, one per warp (NROWS / 8 rows each, one more for
// the first NROWS % 8 warps); for each row r of its band the warp calls emit(r, S, M, N) with rows
// r-1, r, r+1 as produced by load(). The band length is a compile-time constant, so the loop is
// unrolled: the three rows rotate through registers without copies and every row's shared-memory
// address is the band's base plus a constant.
template <int R0, int NROWS, class Load, class Emit>
__device__ __forceinline__ void tm_walk(Load load, Emit emit) {
  constexpr int NW = TM_NT / 32;
  constexpr int PER = NROWS / NW, EXTRA = NROWS % NW;
  static_assert(PER >= 1, "every warp walks at least one row");
  const int warp = threadIdx.x >> 5;
  const int a = R0 + warp * PER + min(warp, EXTRA);
  auto S = load(a - 1);
  auto M = load(a);
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const auto N = load(a + i + 1);
    emit(a + i, S, M, N);
    S = M;
    M = N;
  }
  if (EXTRA > 0 && warp < EXTRA) {
    const auto N = load(a + PER + 1);
    emit(a + PER, S, M, N);
  }
}

// Zero the points of a stage's output row that lie outside the grid (tiles at the grid's edge).
__device__ __forceinline__ void tm_mask(float (&o)[4], int gx0, int gy, int n) {
  const int gx = gx0 + 4 * (threadIdx.x & 31);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((unsigned)gy >= (unsigned)n || (unsigned)(gx + k) >= (unsigned)n) o[k] = 0.f;
}

// This lane's four columns of the tile's output rows in a global array, set up once per tile:
// lanes 1..30 own the output columns; `full` lanes store float4 rows, the lane holding the grid's
// last columns stores them one by one.
struct TmColumn {
  float* p;       // column gx of row 0
  int ld, n, cols;  // cols: columns of the four this lane stores (0: none)
  __device__ __forceinline__ TmColumn(float* base, int ld_, int gx0, int n_) : ld(ld_), n(n_) {
    const int lane = threadIdx.x & 31, gx = gx0 + 4 * lane;
    cols = (lane >= 1 && lane <= 30 && gx < n_) ? min(4, n_ - gx) : 0;
    p = base + gx;
  }
  // A tile away from the grid's edges: lanes 1..30 store whole float4 rows (pred folds in the row
  // and lane conditions, so the store is one predicated instruction)
  __device__ __forceinline__ void store_inner(int gy, const float (&o)[4], bool pred) const {
    if (pred) *reinterpret_cast<float4*>(p + gy * ld) = make_float4(o[0], o[1], o[2], o[3]);
  }
  __device__ __forceinline__ void store(int gy, const float (&o)[4]) const {
    if (gy >= n || cols == 0) return;
    float* q = p + gy * ld;
    if (cols == 4) {
      *reinterpret_cast<float4*>(q) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
      q[0] = o[0];
      if (cols > 1) q[1] = o[1];
      if (cols > 2) q[2] = o[2];
    }
  }
};

// The tiles a persistent CTA visits: tile blockIdx.x, then every gridDim.x-th one, in row-major
// order of tiles_x tiles per row; coordinates advance incrementally (no division per tile).
struct TmTiles {
  int nx, ny, x0, y0, dx, dy;
  __device__ __forceinline__ TmTiles(int tiles_x, int tiles)
      : nx(tiles_x), ny(tiles / tiles_x), x0((int)blockIdx.x % tiles_x), y0((int)blockIdx.x / tiles_x),
        dx((int)gridDim.x % tiles_x), dy((int)gridDim.x / tiles_x) {}
  __device__ __forceinline__ void advance(int& x, int& y) const {
    x += dx;
    y += dy;
    if (x >= nx) {
      x -= nx;
      ++y;
    }
  }
};

// The four points of a lane at once, with the Blackwell paired FP32 instructions (two lanes of
// arithmetic per instruction, each element rounded as the scalar operation would be, so the results
// equal jacobi_update / residual_at bit for bit): the neighbour pair sums are scalar additions, the
// multiply-add chain runs on the pairs (points 0,1 and 2,3).
struct Coef2 {
  float2 w, b0, bwe, bns, bnw, bne, c0, cwe, cns, cnw, cne;  // both halves the same coefficient
  __device__ __forceinline__ explicit Coef2(const Coef<float>& c)
      : w(make_float2(c.w, c.w)), b0(make_float2(c.b0, c.b0)), bwe(make_float2(c.bwe, c.bwe)),
        bns(make_float2(c.bns, c.bns)), bnw(make_float2(c.bnw, c.bnw)), bne(make_float2(c.bne, c.bne)),
        c0(make_float2(-c.c0, -c.c0)), cwe(make_float2(-c.cwe, -c.cwe)), cns(make_float2(-c.cns, -c.cns)),
        cnw(make_float2(-c.cnw, -c.cnw)), cne(make_float2(-c.cne, -c.cne)) {}
};

template <bool RES>
__device__ __forceinline__ void stencil4(const Row6& S, const Row6& M, const Row6& N, const float (&f)[4],
                                         const Coef2& c, float (&o)[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = 2 * h;
    const Nb<float> a = nb6(S, M, N, k), b = nb6(S, M, N, k + 1);
    const float2 cc = make_float2(a.c, b.c), ff = make_float2(f[k], f[k + 1]);
    const float2 we = make_float2(a.we, b.we), ns = make_float2(a.ns, b.ns);
    const float2 d1 = make_float2(a.d1, b.d1), d2 = make_float2(a.d2, b.d2);
    float2 t;
    if (RES) {  // f - A v, in residual_at's order
      t = __ffma2_rn(c.c0, cc, ff);
      t = __ffma2_rn(c.cwe, we, t);
      t = __ffma2_rn(c.cns, ns, t);
      t = __ffma2_rn(c.cnw, d1, t);
      t = __ffma2_rn(c.cne, d2, t);
    } else {    // damped Jacobi, in jacobi_update's order
      t = __fmul2_rn(c.b0, cc);
      t = __ffma2_rn(c.w, ff, t);
      t = __ffma2_rn(c.bwe, we, t);
      t = __ffma2_rn(c.bns, ns, t);
      t = __ffma2_rn(c.bnw, d1, t);
      t = __ffma2_rn(c.bne, d2, t);
    }
    o[k] = t.x;
    o[k + 1] = t.y;
  }
}

// A row of the zero-start walk: v1 = w f with its halo, and the f row itself.
struct ZRow {
  Row6 v;
  float f[4];
};

struct TmaPassArgs {
  int n, ty, tiles_x, tiles;  // grid side, output rows per tile, tiles per row of tiles, all tiles
  int level;
  const float* coef;
  const int* skip;
  int* err;                   // set to TM_ERR_TIMEOUT when a copy never completes
  int stall_tile;             // pass A test hook: this tile's copies are never issued (-1: none)
  float* vout;                // pass A: relaxed v (nullable); pass B: corrected and relaxed v
  int ldvout;
  float* fc;                  // pass A: coarse right-hand side
  int ldc;
};

// Every thread's verdict on a bounded wait, agreed across the CTA (a barrier all threads reach).
__device__ __forceinline__ bool tm_wait_all(uint64_t* bar, uint32_t parity) {
  const bool ok = mbar_wait_bounded(bar, parity);
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// On a timed-out wait: report, then let the copies this CTA still has in flight land (bounded)
// before the CTA's shared memory is released.
__device__ __forceinline__ void tm_abort(int* err, uint64_t* bars, uint32_t pending_parity, uint32_t pending) {
  if (threadIdx.x == 0 && err) atomicExch(err, TM_ERR_TIMEOUT);
  for (int s = 0; s < 2; ++s)
    if ((pending >> s) & 1u) (void)mbar_wait_bounded(bars + s, (pending_parity >> s) & 1u);
}

// ------------------------------------------------------------------------------------------------
// Pass A: nu = 2 damped-Jacobi sweeps (ZERO: from v = 0), residual, full weighting.
// ------------------------------------------------------------------------------------------------
template <bool ZERO, int TY>
__global__ void __launch_bounds__(TM_NT, 3)
    pass_a_tma32(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_f,
                 const TmaPassArgs a) {
  if (a.skip && *a.skip) return;
  constexpr int NU = 2;
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* smem_raw = tm_base(smem_dyn);
  constexpr int R = tm_rows_a(TY, NU);
  constexpr size_t FB = tm_field_a(TY, NU);
  // buffer set s: f at set(s), v (not from zero) one field after it
  const size_t SET = (ZERO ? 1 : 2) * FB;
  auto fin = [&](int s) { return reinterpret_cast<float*>(smem_raw + s * SET); };
  auto vin = [&](int s) { return reinterpret_cast<float*>(smem_raw + s * SET + FB); };
  unsigned char* p = smem_raw + 2 * SET;
  float* work = reinterpret_cast<float*>(p); p += FB;
  float2* hsum = reinterpret_cast<float2*>(p); p += tm_align(size_t(64) * R * 4);
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);

  const int n = a.n, nc = (n - 1) / 2, lane = threadIdx.x & 31;
  const bool inner = (unsigned)(lane - 1) < 30u;  // lanes holding output columns
  const uint32_t box_bytes = (uint32_t)(TM_P * R * 4) * (ZERO ? 1u : 2u);
  const Coef<float> c = load_coef(a.coef, a.level);
  const Coef2 c2(c);
  if (threadIdx.x == 0) {
    prefetch_tensormap(&map_f);
    if (!ZERO) prefetch_tensormap(&map_v);
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t pending = 0u, pend_par = 0u;  // bit s: copies into set s in flight, and their phase parity
  auto issue = [&](int bx, int by, int s, uint32_t parity) {
    if (threadIdx.x == 0) {
      const int gx0 = bx * TM_TX - TM_HX, gy0 = by * TY - (NU + 2);
      mbar_expect_tx(bars + s, box_bytes);
      if (by * a.tiles_x + bx != a.stall_tile) {
        tma_load_2d(fin(s), &map_f, bars + s, gx0, gy0);
        if (!ZERO) tma_load_2d(vin(s), &map_v, bars + s, gx0, gy0);
      }
    }
    pending |= 1u << s;
    pend_par = (pend_par & ~(1u << s)) | (parity << s);
  };
  TmTiles tl(a.tiles_x, a.tiles);
  int bx = tl.x0, by = tl.y0, px = bx, py = by;  // this CTA's current tile, and the next to fetch
  if (by < tl.ny) issue(px, py, 0, 0u);
  tl.advance(px, py);
  for (int it = 0; by < tl.ny; ++it, tl.advance(bx, by)) {
    const int s = it & 1;
    if (!tm_wait_all(bars + s, (uint32_t)(it >> 1) & 1u)) {
      tm_abort(a.err, bars, pend_par, pending);
      return;
    }
    pending &= ~(1u << s);
    // past this barrier every thread has finished the previous tile, whose buffer set the copies of
    // the next tile refill
    if (py < tl.ny) issue(px, py, s ^ 1, (uint32_t)((it + 1) >> 1) & 1u);
    tl.advance(px, py);
    const int x0 = bx * TM_TX, y0 = by * TY;
    const int gx0 = x0 - TM_HX, gy0 = y0 - (NU + 2);
    const bool edge = gx0 < 0 || gy0 < 0 || gx0 + TM_P > n || gy0 + R > n;
    // tiles away from the grid's edges (all but a few percent) run without masks and with
    // predicated whole-row stores; the edge tiles take the general code
    auto tile = [&](auto edge_c) {
    constexpr bool EDGE = decltype(edge_c)::value;
    const float* fs = fin(s);
    float* v2;  // the second sweep's result
    if (ZERO) {
      // sweep 2 from v1 = w f on rows [2, R - 2): v1 formed in registers from the f rows
      // (each f row is read once: the window carries it beside v1)
      tm_walk<2, R - 4>(
              [&](int r) {
                ZRow z;
                tm_f4(fs, r, z.f);
                float q[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) q[k] = c.w * z.f[k];
                z.v = with_halo(q);
                return z;
              },
              [&](int r, const ZRow& S, const ZRow& M, const ZRow& N) {
                float o[4];
                stencil4<false>(S.v, M.v, N.v, M.f, c2, o);
                if constexpr (EDGE) tm_mask(o, gx0, gy0 + r, n);
                tm_st4(work, r, o);
              });
      v2 = work;
    } else {
      float* vs = vin(s);
      tm_walk<1, R - 2>([&](int r) { return tm_row(vs, r); },
              [&](int r, const Row6& S, const Row6& M, const Row6& N) {
                float fv[4], o[4];
                tm_f4(fs, r, fv);
                stencil4<false>(S, M, N, fv, c2, o);
                if constexpr (EDGE) tm_mask(o, gx0, gy0 + r, n);
                tm_st4(work, r, o);
              });
      __syncthreads();
      tm_walk<2, R - 4>([&](int r) { return tm_row(work, r); },
              [&](int r, const Row6& S, const Row6& M, const Row6& N) {
                float fv[4], o[4];
                tm_f4(fs, r, fv);
                stencil4<false>(S, M, N, fv, c2, o);
                if constexpr (EDGE) tm_mask(o, gx0, gy0 + r, n);
                tm_st4(vs, r, o);
              });
      v2 = vs;
    }
    __syncthreads();
    // residual on rows [3, R - 3) (full weighting of the output rows reads one row beyond them);
    // the relaxed v of the output rows [4, R - 4) goes to global memory from the same registers
    const TmColumn out(a.vout, a.ldvout, gx0, n);
    tm_walk<3, R - 6>([&](int r) { return tm_row(v2, r); },
            [&](int r, const Row6& S, const Row6& M, const Row6& N) {
              float fv[4], res[4];
              tm_f4(fs, r, fv);
              stencil4<true>(S, M, N, fv, c2, res);
              const float nxt = __shfl_down_sync(0xffffffffu, res[0], 1);
              float2 h;
              h.x = fmaf(2.f, res[1], res[0] + res[2]);
              h.y = fmaf(2.f, res[3], res[2] + nxt);
              hsum[r * 32 + lane] = h;
              const float o[4] = {M.v[0], M.v[1], M.v[2], M.v[3]};
              if constexpr (EDGE) {
                if (r >= NU + 2 && r < R - (NU + 2)) out.store(gy0 + r, o);
              } else {
                out.store_inner(gy0 + r, o, inner && r >= NU + 2 && r < R - (NU + 2));
              }
            });
    __syncthreads();
    // coarse point (I, J) on fine (2I+1, 2J+1): staged row 2j + 5 for j = J - y0/2, staged columns
    // 4q + 1 and 4q + 3 of lane q (I = x0/2 + 2q - 2 and the next)
    {
      constexpr int NW = TM_NT / 32;
      constexpr int cj_n = TY / 2;
      const int I = x0 / 2 + 2 * lane - 2;
      const int ccols = EDGE ? ((lane >= 1 && lane <= 30 && I < nc) ? min(2, nc - I) : 0) : (inner ? 2 : 0);
      float* cp = a.fc + I;
      for (int j = threadIdx.x >> 5; j < cj_n; j += NW) {
        const int J = y0 / 2 + j;
        const int r = 2 * j + (NU + 2) + 1;
        const float2 hs = hsum[(r - 1) * 32 + lane], hm = hsum[r * 32 + lane], hn = hsum[(r + 1) * 32 + lane];
        if (ccols && (!EDGE || J < nc)) {
          float2 o;
          o.x = 0.0625f * fmaf(2.f, hm.x, hs.x + hn.x);
          o.y = 0.0625f * fmaf(2.f, hm.y, hs.y + hn.y);
          float* q = cp + J * a.ldc;
          if (ccols == 2) *reinterpret_cast<float2*>(q) = o;
          else q[0] = o.x;
        }
      }
    }
    };
    if (edge) tile(std::true_type{});
    else tile(std::false_type{});
    // this tile's generic-proxy writes to buffer set s are ordered before the tensor copies that
    // refill it (issued after the next tile's wait, whose barrier every thread passes first)
    fence_proxy_async_smem();
  }
}

// ------------------------------------------------------------------------------------------------
// Pass B: v <- v + P v_c (bilinear), nu = 2 damped-Jacobi sweeps.
// ------------------------------------------------------------------------------------------------
template <int TY>
__global__ void __launch_bounds__(TM_NT, 2)
    pass_b_tma32(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_f,
                 const __grid_constant__ CUtensorMap map_c, const TmaPassArgs a) {
  if (a.skip && *a.skip) return;
  constexpr int NU = 2;
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* smem_raw = tm_base(smem_dyn);
  constexpr int R = tm_rows_b(TY, NU), CR = tm_crows_b(TY, NU);
  constexpr size_t FB = tm_field_b(TY, NU), CB = tm_cfield_b(TY, NU);
  // buffer set s: v, f, then the coarse window
  const size_t SET = 2 * FB + CB;
  auto vin = [&](int s) { return reinterpret_cast<float*>(smem_raw + s * SET); };
  auto fin = [&](int s) { return reinterpret_cast<float*>(smem_raw + s * SET + FB); };
  auto cin = [&](int s) { return reinterpret_cast<float*>(smem_raw + s * SET + 2 * FB); };
  unsigned char* p = smem_raw + 2 * SET;
  float* work = reinterpret_cast<float*>(p); p += FB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);

  const int n = a.n, lane = threadIdx.x & 31;
  const bool inner = (unsigned)(lane - 1) < 30u;  // lanes holding output columns
  const uint32_t box_bytes = (uint32_t)(2 * TM_P * R * 4 + TM_CP * CR * 4);
  const Coef<float> c = load_coef(a.coef, a.level);
  const Coef2 c2(c);
  if (threadIdx.x == 0) {
    prefetch_tensormap(&map_v);
    prefetch_tensormap(&map_f);
    prefetch_tensormap(&map_c);
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t pending = 0u, pend_par = 0u;  // bit s: copies into set s in flight, and their phase parity
  // window origin: fine (gx0, gy0) = (x0 - 4, y0 - NU); coarse (cx0, cy0) with cx0 = x0/2 - 4
  // (x0/2 - 3 rounded down to a multiple of 4, the tensor copy's alignment) and cy0 = gy0/2 - 1
  auto issue = [&](int bx, int by, int s, uint32_t parity) {
    if (threadIdx.x == 0) {
      const int x0 = bx * TM_TX, y0 = by * TY;
      const int gy0 = y0 - NU;
      mbar_expect_tx(bars + s, box_bytes);
      tma_load_2d(vin(s), &map_v, bars + s, x0 - TM_HX, gy0);
      tma_load_2d(fin(s), &map_f, bars + s, x0 - TM_HX, gy0);
      tma_load_2d(cin(s), &map_c, bars + s, x0 / 2 - 4, (gy0 >> 1) - 1);
    }
    pending |= 1u << s;
    pend_par = (pend_par & ~(1u << s)) | (parity << s);
  };
  TmTiles tl(a.tiles_x, a.tiles);
  int bx = tl.x0, by = tl.y0, px = bx, py = by;  // this CTA's current tile, and the next to fetch
  if (by < tl.ny) issue(px, py, 0, 0u);
  tl.advance(px, py);
  for (int it = 0; by < tl.ny; ++it, tl.advance(bx, by)) {
    const int s = it & 1;
    if (!tm_wait_all(bars + s, (uint32_t)(it >> 1) & 1u)) {
      tm_abort(a.err, bars, pend_par, pending);
      return;
    }
    pending &= ~(1u << s);
    if (py < tl.ny) issue(px, py, s ^ 1, (uint32_t)((it + 1) >> 1) & 1u);
    tl.advance(px, py);
    const int x0 = bx * TM_TX, y0 = by * TY;
    const int gx0 = x0 - TM_HX, gy0 = y0 - NU;
    const int cy0 = (gy0 >> 1) - 1;
    const bool edge = gx0 < 0 || gy0 < 0 || gx0 + TM_P > n || gy0 + R > n;
    auto tile = [&](auto edge_c) {  // interior tiles: no masks, predicated whole-row stores
    constexpr bool EDGE = decltype(edge_c)::value;
    const float* vs = vin(s);
    const float* fs = fin(s);
    const float* cs = cin(s);
    // coarse row J interpolated in x to this lane's four fine columns gx0 + 4q .. + 3: fine x even
    // lies between coarse x/2 - 1 and x/2, odd x on coarse (x - 1)/2; in the window, coarse x/2 of
    // column 4q is at 2q + 2 (the window starts at x0/2 - 4 = gx0/2 - 2)
    auto coarse_x = [&](int J, float (&o)[4]) {
      const float2 q = *reinterpret_cast<const float2*>(cs + (J - cy0) * TM_CP + 2 * lane + 2);
      const float left = __shfl_up_sync(0xffffffffu, q.y, 1);  // coarse x/2 - 1 (lane 0: a halo column)
      o[0] = 0.5f * (left + q.x);
      o[1] = q.x;
      o[2] = 0.5f * (q.x + q.y);
      o[3] = q.y;
    };
    // sweep 1 on rows [1, R - 1) from the corrected v = v + P v_c, formed as rows enter the window
    tm_walk<1, R - 2>(
            [&](int r) {
              float v[4], ca[4];
              tm_f4(vs, r, v);
              const int gy = gy0 + r;
              if (gy & 1) {
                coarse_x((gy - 1) >> 1, ca);
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] += ca[k];
              } else {
                float cb[4];
                coarse_x((gy >> 1) - 1, ca);
                coarse_x(gy >> 1, cb);
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] += 0.5f * (ca[k] + cb[k]);
              }
              if constexpr (EDGE) tm_mask(v, gx0, gy, n);
              return with_halo(v);
            },
            [&](int r, const Row6& S, const Row6& M, const Row6& N) {
              float fv[4], o[4];
              tm_f4(fs, r, fv);
              stencil4<false>(S, M, N, fv, c2, o);
              if constexpr (EDGE) tm_mask(o, gx0, gy0 + r, n);
              tm_st4(work, r, o);
            });
    __syncthreads();
    // sweep 2 on the output rows [2, R - 2), written to global memory
    const TmColumn out(a.vout, a.ldvout, gx0, n);
    tm_walk<NU, R - 2 * NU>([&](int r) { return tm_row(work, r); },
            [&](int r, const Row6& S, const Row6& M, const Row6& N) {
              float fv[4], o[4];
              tm_f4(fs, r, fv);
              stencil4<false>(S, M, N, fv, c2, o);
              if constexpr (EDGE) out.store(gy0 + r, o);
              else out.store_inner(gy0 + r, o, inner);
            });
    };
    if (edge) tile(std::true_type{});
    else tile(std::false_type{});
    // this tile's generic-proxy writes to buffer set s are ordered before the tensor copies that
    // refill it (issued after the next tile's wait, whose barrier every thread passes first)
    fence_proxy_async_smem();
  }
}

}  // namespace kc
