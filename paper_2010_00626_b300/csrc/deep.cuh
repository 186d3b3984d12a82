// Persistent deep calls: one call at a small level with everything below it in one cooperative
// launch (Algorithm 3's recursion walked on the device by every CTA of the grid in lock step).
//
// Below a few hundred points per side a level's pass is a few microseconds of latency-bound work,
// and a kappa-cycle makes hundreds of such calls (the sum of Prop. 2.2's counts over the small
// levels); as separate launches each pays its launch and its ramp. Here a grid of co-resident CTAs
// (a cooperative launch: one or two per SM) runs, for the call at level `top` and recursively for
// its child calls, pass A over the level's tiles, a grid barrier, the child calls, pass B over the
// tiles, a grid barrier. At the level just above the coarse kernel's, the two child calls are the
// condensed map v_lc = P_c f_lc (children_matvec), its rows dealt over the whole grid; each CTA's
// rows of P_c arrive in its shared memory by one bulk copy issued before the parent's pass A, so the
// product waits only for f_lc (maps with more rows per CTA than shared memory holds are read from
// global memory instead, asked of L2 at the same point). The last child call's pass B there runs
// inside its parent's pass B (deep_tiles_b2), and in FP32 a first child's pass B with the second
// child's pass A (deep_tiles_ba): one phase and grid barrier fewer each. Every point's
// arithmetic is that of the separate launches (the same tile functions on the same tiles, the same
// per-row sums), so the results equal them bit for bit.
//
// The grid barrier: after a CTA barrier, one thread per CTA counts the CTA in with an acquire-release
// atomic add and polls the count with acquire loads until the whole grid has arrived (release and
// acquire at GPU scope order every write before the barrier, of any thread of the CTA, before every
// read after it). Waits are bounded (half a second of the global timer): a CTA whose wait runs out
// records DEEP_ERR_TIMEOUT and returns, so every other CTA's next wait runs out too; the host
// reports MG_ERR_TIMEOUT and clears the barrier words.
#pragma once
#include <stdint.h>

#include "kernels.cuh"
#include "tma_f32.cuh"  // mbarrier helpers and bounded waits

namespace kc {

constexpr int DEEP_MAX_DEPTH = 6;                   // levels whose passes one launch runs
constexpr uint64_t GRID_WAIT_NS = 500000000ull;     // a grid barrier waits at most half a second
constexpr uint32_t GRID_WAIT_POLLS = 1u << 26;      // and at most this many polls
constexpr int DEEP_ERR_TIMEOUT = 2;

template <typename T>
struct DeepArgs {
  PassAArgs<T> pa[DEEP_MAX_DEPTH];  // level top + d; the kernel clears vin for a zero start
  PassBArgs<T> pb[DEEP_MAX_DEPTH];
  int tile[DEEP_MAX_DEPTH];         // tile edge of level top + d (8, 16 or 32), as its separate launches
  CoarseArgs<T> cc;                 // the condensed level lc = top + depth: v, f, their pitches, side
  const T* pmap;                    // P of counter class 1; class c at pmap + (c - 1) * pstride
  size_t pstride;
  int pld, pcls;
  int top, depth;
  int kappa, zero;                  // the launch's call: counter and start
  int prow_off;                     // shared-memory offset of the staged rows of P (16-byte aligned)
  int staged;                       // 1: P's rows staged in shared memory; 0: read from global memory
                                    // (asked of L2 ahead), for maps too large to stage
  int stall_cta;                    // test hook: this CTA leaves at once (-1: none)
  int merge_b;                      // 1: the last child call's pass B at the level above the condensed one
                                    // runs inside its parent's pass B (8 x 8 parent tiles, nu2 = 2)
  int merge_ba;                     // 1: there, a first child's pass B and the second child's pass A run
                                    // as one phase (8 x 8 tiles, nu1 = nu2 = 2)
  unsigned* bar;                    // grid barrier words: arrivals, exits (both zero at rest)
  int* err;                         // set to DEEP_ERR_TIMEOUT when a barrier wait runs out
  const int* skip;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t deep_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// All CTAs of the grid meet; false (in every thread of the CTA) when this CTA's wait ran out. The
// arrival is one acquire-release add on the count; a CTA that is not the last of its generation
// polls the count with acquire loads until it reaches the generation's end (count a multiple of
// the grid size: deep_exit clears it when the launch ends).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int good;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    const unsigned target = (old / gridDim.x + 1u) * gridDim.x;
    if (old + 1u != target) {
      const uint64_t t0 = deep_ns();
      for (uint32_t it = 1; ld_acquire_gpu(bar) < target; ++it) {
        if (it >= GRID_WAIT_POLLS || ((it & 63u) == 0 && deep_ns() - t0 > GRID_WAIT_NS)) {
          ok = 0;
          atomicExch(err, DEEP_ERR_TIMEOUT);
          break;
        }
      }
    }
    good = ok;
  }
  __syncthreads();
  return good != 0;
}

// The end of a launch: the last CTA out (every CTA has passed every barrier by then) clears the
// barrier words for the next launch.
__device__ __forceinline__ void deep_exit(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0 && atomicAdd(bar + 1, 1u) == gridDim.x - 1) {
    atomicExch(bar, 0u);
    atomicExch(bar + 1, 0u);
  }
}

// one point per thread and staging round (fewer registers for the whole kernel; an 8 x 8 tile's
// window fits the CTA in one round anyway)
template <typename T, int B, int NT>
__device__ __forceinline__ void deep_tiles_a(const PassAArgs<T>& pa, unsigned char* smem) {
  const int tx = (pa.n + B - 1) / B, nt = tx * tx;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    pass_a_tile<T, B, B, NT, false, 1>(pa, t % tx, t / tx, 0, smem);
    __syncthreads();  // the next tile reuses the shared memory
  }
}
template <typename T, int B, int NT>
__device__ __forceinline__ void deep_tiles_b(const PassBArgs<T>& pb, unsigned char* smem) {
  const int tx = (pb.n + B - 1) / B, nt = tx * tx;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    pass_b_tile<T, B, B, NT, false, 1>(pb, t % tx, t / tx, 0, smem);
    __syncthreads();
  }
}

// Shared memory of deep_tiles_b2: the parent tile's pass B, then the child window's.
template <typename T>
__host__ __device__ constexpr size_t deep_b2_smem() {
  return ((pass_b_smem<T, 8, 8>(2, false) + 15) / 16) * 16 + pass_b_smem<T, 7, 7>(2, false);
}

// The last child call's pass B (level l+1, args `child`) and its parent's pass B (level l) as one
// phase: for each 8 x 8 parent tile, the child's pass B over the 7 x 7 coarse window that the
// parent's interpolation reads (nu = 2), written straight into the parent's coarse staging buffer
// (zero outside the grid, as the parent would load it), then the parent's pass B from there. The
// child's points are computed by the formula of its own pass, from the same inputs, so the parent
// sees the values a separate child pass would have stored; the child's own result is not needed
// after this point (the next calls at its level start from zero), so it is not stored.
template <typename T, int NT>
__device__ __forceinline__ void deep_tiles_b2(const PassBArgs<T>& child, const PassBArgs<T>& parent,
                                              unsigned char* smem) {
  constexpr int B = 8, CR = 7;
  const int tx = (parent.n + B - 1) / B, nt = tx * tx;
  unsigned char* child_smem = smem + ((pass_b_smem<T, B, B>(2, false) + 15) / 16) * 16;
  T* cs = pass_b_cs<T, B, B>(smem, 2);
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int x0 = (t % tx) * B, y0 = (t / tx) * B;
    // the parent's coarse window starts at (x0 - 2) / 2 - 1 (x0 is even)
    pass_b_core<T, CR, CR, NT, false, 1, PB_TO_SMEM>(child, x0 / 2 - 2, y0 / 2 - 2, 0, child_smem, cs, CR);
    __syncthreads();
    pass_b_core<T, B, B, NT, false, 1, PB_CS_READY>(parent, x0, y0, 0, smem);
    __syncthreads();
  }
}

// Shared memory of deep_tiles_ba: the tile's pass A, then the first child's window pass B.
template <typename T>
__host__ __device__ constexpr size_t deep_ba_smem() {
  return ((pass_a_smem<T, 8, 8>(2) + 15) / 16) * 16 + pass_b_smem<T, 15, 15>(2, false);
}

// A first child call's pass B (args `pb`) and the second child call's pass A (args `pa`, the same
// level, from that result) as one phase: for each 8 x 8 tile, the first child's pass B over the
// 15 x 15 window that pass A stages for v (nu1 = 2: halo 3), written straight into pass A's v
// buffer (zero outside the grid), then pass A from there. Same formulas on the same inputs as the
// two separate passes; the first child's result is needed only by this pass A, so it is not stored.
template <typename T, int NT>
__device__ __forceinline__ void deep_tiles_ba(const PassBArgs<T>& pb, const PassAArgs<T>& pa, unsigned char* smem) {
  constexpr int B = 8, VR = 15;
  const int tx = (pa.n + B - 1) / B, nt = tx * tx;
  unsigned char* b_smem = smem + ((pass_a_smem<T, B, B>(2) + 15) / 16) * 16;
  T* vwin = reinterpret_cast<T*>(smem);  // pass A's first buffer: v's window, pitch 15
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int x0 = (t % tx) * B, y0 = (t / tx) * B;
    pass_b_core<T, VR, VR, NT, false, 1, PB_TO_SMEM>(pb, x0 - 3, y0 - 3, 0, b_smem, vwin, VR);
    __syncthreads();
    pass_a_tile<T, B, B, NT, false, 1, true>(pa, t % tx, t / tx, 0, smem);
    __syncthreads();
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) deep_kernel(const DeepArgs<T> a) {
  if (a.skip && *a.skip) return;  // the same flag for every CTA: the whole grid returns
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // this CTA's rows of P (a contiguous block, see child_rows_lo) and the copy's barrier after them
  const int S = a.cc.n_lc * a.cc.n_lc;
  const int rlo = child_rows_lo(S, blockIdx.x, gridDim.x), rhi = child_rows_lo(S, blockIdx.x + 1, gridDim.x);
  T* prow = reinterpret_cast<T*>(smem_raw + a.prow_off);
  const uint32_t pbytes = a.staged ? (uint32_t)((size_t)(rhi - rlo) * a.pld * sizeof(T)) : 0u;
  uint64_t* pbar = reinterpret_cast<uint64_t*>(smem_raw + a.prow_off + (((size_t)pbytes + 15) & ~(size_t)15));
  uint32_t pphase = 0;
  bool pinflight = false;
  if (threadIdx.x == 0 && pbytes) {
    mbar_init(pbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if ((int)blockIdx.x == a.stall_cta) return;  // the others' first barrier wait runs out
  // a CTA whose barrier wait ran out lets its copy of P's rows land (bounded) before it leaves
  auto bail = [&]() {
    if (pinflight) (void)mbar_wait_bounded(pbar, pphase);
  };
  // before the pass A of a call whose children are condensed (counter k): this CTA's rows of P_c
  // into shared memory by one bulk copy, or (unstaged maps) asked of L2
  auto fetch_p = [&](int k) {
    const int c = k < a.pcls ? k : a.pcls;
    const T* rows = a.pmap + (size_t)(c - 1) * a.pstride;
    if (!a.staged) {
      children_prefetch(rows, a.pld, S, blockIdx.x, gridDim.x);
    } else if (pbytes) {
      if (threadIdx.x == 0) {
        // the previous product's reads of the rows (before a CTA barrier) precede this refill
        fence_proxy_async_smem();
        mbar_expect_tx(pbar, pbytes);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(prow)), "l"(rows + (size_t)rlo * a.pld), "r"(pbytes), "r"(smem_u32(pbar))
                     : "memory");
      }
      pinflight = true;
    }
  };
  // the recursion's frames: counter, start and stage of the call at depth d (level top + d)
  int kap[DEEP_MAX_DEPTH], zer[DEEP_MAX_DEPTH], stage[DEEP_MAX_DEPTH];
  int d = 0;
  kap[0] = a.kappa;
  zer[0] = a.zero;
  stage[0] = 0;
  while (d >= 0) {
    if (stage[d] == 0 || stage[d] == 4) {  // pass A (stage 4: already run), then the child calls
      if (stage[d] == 0) {
        if (d + 1 == a.depth) fetch_p(kap[d]);
        PassAArgs<T> pa = a.pa[d];
        if (zer[d]) pa.vin = nullptr;
        switch (a.tile[d]) {
          case 32: deep_tiles_a<T, 32, NT>(pa, smem_raw); break;
          case 16: deep_tiles_a<T, 16, NT>(pa, smem_raw); break;
          default: deep_tiles_a<T, 8, NT>(pa, smem_raw); break;
        }
        if (!grid_barrier(a.bar, a.err)) return bail();
      }
      if (d + 1 == a.depth) {  // children at the coarse-kernel level: v_lc = P_c f_lc
        if (pinflight) {
          if (!tm_wait_all(pbar, pphase)) {
            if (threadIdx.x == 0) atomicExch(a.err, DEEP_ERR_TIMEOUT);
            (void)mbar_wait_bounded(pbar, pphase);  // let the copy land before the CTA leaves
            return;
          }
          pphase ^= 1u;
          pinflight = false;
        }
        if (a.staged) {
          children_matvec<T, NT, 1, 8, true>(nullptr, a.pld, a.cc, blockIdx.x, gridDim.x,
                                             reinterpret_cast<T*>(smem_raw), prow);
        } else {
          const int c = kap[d] < a.pcls ? kap[d] : a.pcls;
          children_matvec<T, NT, 1, 8>(a.pmap + (size_t)(c - 1) * a.pstride, a.pld, a.cc, blockIdx.x, gridDim.x,
                                       reinterpret_cast<T*>(smem_raw));
        }
        if (!grid_barrier(a.bar, a.err)) return bail();
        stage[d] = 3;
      } else {  // first child: counter k from zero
        stage[d] = 1;
        kap[d + 1] = kap[d];
        zer[d + 1] = 1;
        stage[d + 1] = 0;
        ++d;
        continue;
      }
    } else if (stage[d] == 1) {  // second child: counter k - 1 from the first child's result
      if (kap[d] > 1) {
        stage[d] = 2;
        kap[d + 1] = kap[d] - 1;
        zer[d + 1] = 0;
        stage[d + 1] = 0;
        ++d;
        continue;
      }
      stage[d] = 3;
    } else if (stage[d] == 2) {
      stage[d] = 3;
    }
    // stage 3: pass B; the top call's needs no barrier after it (the launch ends)
    if (a.merge_ba && d + 1 == a.depth && d >= 1 && stage[d - 1] == 1 && kap[d - 1] > 1) {
      // a first child with a second to come: its pass B and the second child's pass A in one phase;
      // the second child then continues after its pass A (stage 4) in the same frame
      fetch_p(kap[d - 1] - 1);
      deep_tiles_ba<T, NT>(a.pb[d], a.pa[d], smem_raw);
      if (!grid_barrier(a.bar, a.err)) return bail();
      stage[d - 1] = 2;
      kap[d] = kap[d - 1] - 1;
      zer[d] = 0;
      stage[d] = 4;
      continue;
    }
    if (a.merge_b && d + 1 == a.depth && d >= 1 && (stage[d - 1] == 2 || (stage[d - 1] == 1 && kap[d - 1] <= 1))) {
      // the last child of its parent: both pass B in one phase, and the parent's call is done
      deep_tiles_b2<T, NT>(a.pb[d], a.pb[d - 1], smem_raw);
      if (d > 1 && !grid_barrier(a.bar, a.err)) return bail();
      d -= 2;
      continue;
    }
    switch (a.tile[d]) {
      case 32: deep_tiles_b<T, 32, NT>(a.pb[d], smem_raw); break;
      case 16: deep_tiles_b<T, 16, NT>(a.pb[d], smem_raw); break;
      default: deep_tiles_b<T, 8, NT>(a.pb[d], smem_raw); break;
    }
    if (d > 0 && !grid_barrier(a.bar, a.err)) return bail();
    --d;
  }
  deep_exit(a.bar);
}

}  // namespace kc
