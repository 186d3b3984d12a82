// Device kernels of the kappa-cycle multigrid (Avnat & Yavneh, arXiv 2010.00626) for sm_103a.
//
// Grid functions are row-major n x n arrays of interior points with a pitch (ld); element
// (i, j) -- i the x index, j the y index, j+1 north -- is at [j*ld + i]. Dirichlet boundary
// values are zero and never stored; every kernel treats points outside [0,n)^2 as zero.
//
// Level kernels (one launch per level visit, Section 2.1 / Algorithm 3):
//   pass_a_kernel   relax nu1 times + residual + full-weighting restriction, fused in one
//                   shared-memory tile (temporal blocking: the tile carries a halo of nu1+1
//                   points and recomputes the shrinking halo, so v and f are read once and the
//                   relaxed v and the coarse right-hand side are written once).
//   pass_b_kernel   bilinear interpolation + correction + relax nu2 times (+ optional partial
//                   sums of ||f - A v||^2 for the stopping test), fused the same way.
//   coarse_kernel   one CTA that keeps every level at or below a small grid side in shared
//                   memory and walks the kappa recursion itself (an explicit stack), so the
//                   many sequential coarse-level calls cost no kernel launches.
// All level arithmetic is done in T (double on the FP64 path); norms and dot products always
// accumulate in double.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kc {

constexpr int MAXL = 16;

// Per-level coefficient table (NCOEF entries of type T per level).
// A constant symmetric nine-point stencil has five distinct values: centre c0, west/east cwe,
// south/north cns, north-west/south-east cnw and north-east/south-west cne.
// Damped Jacobi v <- v + w (f - A v), w = omega/c0, is evaluated as
//   b0 v + w f + bwe (vW+vE) + bns (vS+vN) + bnw (vNW+vSE) + bne (vNE+vSW)
// with b0 = 1 - w c0 and b* = -w c*: 4 additions, 1 multiply and 5 multiply-adds per point.
enum {
  C_C0 = 0, C_WE, C_NS, C_NW, C_NE, C_W, C_B0, C_BWE, C_BNS, C_BNW, C_BNE,
  C_ST = 12,  // 9 entries: full stencil st[(dy+1)*3 + (dx+1)] as computed
  NCOEF = 24
};

template <typename T>
struct Coef {
  T c0, cwe, cns, cnw, cne, w, b0, bwe, bns, bnw, bne;
};

template <typename T>
__device__ __forceinline__ Coef<T> load_coef(const T* __restrict__ tab, int level) {
  const T* p = tab + level * NCOEF;
  Coef<T> c;
  c.c0 = p[C_C0]; c.cwe = p[C_WE]; c.cns = p[C_NS]; c.cnw = p[C_NW]; c.cne = p[C_NE];
  c.w = p[C_W]; c.b0 = p[C_B0]; c.bwe = p[C_BWE]; c.bns = p[C_BNS]; c.bnw = p[C_BNW]; c.bne = p[C_BNE];
  return c;
}

// Neighbour sums at position k of a row-major buffer with row stride W (k+W is north).
template <typename T>
struct Nb {
  T c, we, ns, d1, d2;
};
template <typename T>
__device__ __forceinline__ Nb<T> neighbours(const T* s, int k, int W) {
  Nb<T> r;
  r.c = s[k];
  r.we = s[k - 1] + s[k + 1];
  r.ns = s[k - W] + s[k + W];
  r.d1 = s[k + W - 1] + s[k - W + 1];  // NW + SE
  r.d2 = s[k + W + 1] + s[k - W - 1];  // NE + SW
  return r;
}

// One damped-Jacobi update of the point with neighbourhood nb and right-hand side fv.
template <typename T>
__device__ __forceinline__ T jacobi_update(const Nb<T>& nb, T fv, const Coef<T>& c) {
  T t = c.b0 * nb.c;
  t = fma(c.w, fv, t);
  t = fma(c.bwe, nb.we, t);
  t = fma(c.bns, nb.ns, t);
  t = fma(c.bnw, nb.d1, t);
  t = fma(c.bne, nb.d2, t);
  return t;
}

// Residual f - A v at the point.
template <typename T>
__device__ __forceinline__ T residual_at(const Nb<T>& nb, T fv, const Coef<T>& c) {
  T t = fma(-c.c0, nb.c, fv);
  t = fma(-c.cwe, nb.we, t);
  t = fma(-c.cns, nb.ns, t);
  t = fma(-c.cnw, nb.d1, t);
  t = fma(-c.cne, nb.d2, t);
  return t;
}

// (A v) at the point.
template <typename T>
__device__ __forceinline__ T apply_at(const Nb<T>& nb, const Coef<T>& c) {
  T t = c.c0 * nb.c;
  t = fma(c.cwe, nb.we, t);
  t = fma(c.cns, nb.ns, t);
  t = fma(c.cnw, nb.d1, t);
  t = fma(c.cne, nb.d2, t);
  return t;
}

// The stencil operations of the level kernels, for a symmetric stencil (pair sums, NS = false)
// or a general one (NS = true: the non-symmetric convection-diffusion operator, every entry
// separately; the same count of FP64 operations, the pair additions become multiply-adds).
template <typename T, bool NS>
struct StencilOp;

template <typename T>
struct StencilOp<T, false> {
  Coef<T> c;
  __device__ __forceinline__ void load(const T* __restrict__ tab, int level) { c = load_coef(tab, level); }
  __device__ __forceinline__ T w() const { return c.w; }
  __device__ __forceinline__ T jac(const T* s, int k, int W, T fv) const { return jacobi_update(neighbours(s, k, W), fv, c); }
  __device__ __forceinline__ T res(const T* s, int k, int W, T fv) const { return residual_at(neighbours(s, k, W), fv, c); }
  __device__ __forceinline__ T app(const T* s, int k, int W) const { return apply_at(neighbours(s, k, W), c); }
};

template <typename T>
struct StencilOp<T, true> {
  T wv, b0, st[9], b[9];  // b[q] = -w st[q]; st[(dy+1)*3 + (dx+1)] multiplies v[j+dy][i+dx]
  __device__ __forceinline__ void load(const T* __restrict__ tab, int level) {
    const T* p = tab + level * NCOEF;
    wv = p[C_W];
    b0 = p[C_B0];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      st[q] = p[C_ST + q];
      b[q] = -wv * st[q];
    }
  }
  __device__ __forceinline__ T w() const { return wv; }
  __device__ __forceinline__ T jac(const T* s, int k, int W, T fv) const {
    T t = b0 * s[k];
    t = fma(wv, fv, t);
#pragma unroll
    for (int q = 0; q < 9; ++q)
      if (q != 4) t = fma(b[q], s[k + (q / 3 - 1) * W + (q % 3 - 1)], t);
    return t;
  }
  __device__ __forceinline__ T res(const T* s, int k, int W, T fv) const {
    T t = fv;
#pragma unroll
    for (int q = 0; q < 9; ++q) t = fma(-st[q], s[k + (q / 3 - 1) * W + (q % 3 - 1)], t);
    return t;
  }
  __device__ __forceinline__ T app(const T* s, int k, int W) const {
    T t = st[4] * s[k];
#pragma unroll
    for (int q = 0; q < 9; ++q)
      if (q != 4) t = fma(st[q], s[k + (q / 3 - 1) * W + (q % 3 - 1)], t);
    return t;
  }
};

// Full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] of r around position k (row stride W).
template <typename T>
__device__ __forceinline__ T full_weight(const T* r, int k, int W) {
  T e = (r[k - 1] + r[k + 1]) + (r[k - W] + r[k + W]);
  T d = (r[k - W - 1] + r[k - W + 1]) + (r[k + W - 1] + r[k + W + 1]);
  T t = T(0.25) * r[k];
  t = fma(T(0.125), e, t);
  return fma(T(0.0625), d, t);
}

// Visit every point of an Rw x Rh region with NT threads, lanes on consecutive x.
template <int NT, typename F>
__device__ __forceinline__ void for_region(int Rw, int Rh, F fn) {
  const int q = NT / Rw, r = NT - q * Rw;
  int ly = threadIdx.x / Rw, lx = threadIdx.x - ly * Rw;
  while (ly < Rh) {
    fn(lx, ly);
    lx += r;
    ly += q;
    if (lx >= Rw) { lx -= Rw; ++ly; }
  }
}

// Visit every point of an Rw x Rh region as for_region does, K points per thread at a time: a
// round issues all K loads before any of their stores. (A store waits for its load, so visiting
// one point at a time pays one memory round trip per point a thread visits; the small tiles of the
// latency-bound levels give a thread several.)
template <int NT, int K, typename Load, typename Store>
__device__ __forceinline__ void stage_region(int Rw, int Rh, Load load, Store store) {
  const int q = NT / Rw, r = NT - q * Rw;
  int ly = threadIdx.x / Rw, lx = threadIdx.x - ly * Rw;
  while (ly < Rh) {
    int xs[K], ys[K];
    decltype(load(0, 0)) vals[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      xs[u] = lx;
      ys[u] = ly;
      if (ly < Rh) vals[u] = load(lx, ly);
      lx += r;
      ly += q;
      if (lx >= Rw) {
        lx -= Rw;
        ++ly;
      }
    }
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (ys[u] < Rh) store(xs[u], ys[u], vals[u]);
  }
}

// Points per thread and round of a tile's staging: the region of a BX x BY tile with nu = 2 over
// NT threads, at most 8; the 32- and 64-wide tiles of the larger levels keep one (more registers
// would cost them CTAs per SM, and their many warps per SM hide the loads: measured, 32-wide FP64
// pass B at 1023^2 71.0 -> 72.2 us with four).
template <int BX, int BY, int NT>
constexpr int stage_k() {
  return BX == 32 || BX == 64 ? 1
                              : (((BX + 7) * (BY + 7) + NT - 1) / NT > 8 ? 8 : ((BX + 7) * (BY + 7) + NT - 1) / NT);
}

template <typename T>
struct TwoVals {
  T a, b;
};

__device__ __forceinline__ bool inside(int gx, int gy, int n) {
  return (unsigned)gx < (unsigned)n && (unsigned)gy < (unsigned)n;
}

// Deterministic block sum of one double per thread (fixed order); result valid in thread 0.
// Callers that use `red` again must __syncthreads() first.
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  }
  return s;
}

// ---------------------------------------------------------------------------------------------
// Pass A: relax nu times from v (or from zero), then f_c = R (f - A v) (Algorithm 3, steps 2-4)
// ---------------------------------------------------------------------------------------------
template <typename T>
struct PassAArgs {
  const T* vin;   // nullptr: zero initial guess (the v^{l+1} <- 0 of Algorithm 3)
  T* vout;        // relaxed v (must not alias vin); nullptr: not written
  const T* f;
  T* fc;          // coarse right-hand side, (n-1)/2 square
  const T* coef;
  const int* skip;  // nullable; kernel returns at once when *skip != 0
  double* partial;  // nullable (nu >= 1): per-block sum of squared residuals of vin over the tile,
                    // formed by the first sweep, written as v + w (f - A v)
  int ldvin, ldvout, ldf, ldc;
  int n, nu, level;
};

// Shared memory: two v buffers and f, each (BX+2H+1) x (BY+2H+1), H = nu + 1.
template <typename T, int BX, int BY>
__host__ __device__ constexpr size_t pass_a_smem(int nu) {
  return size_t(3) * (BX + 2 * (nu + 1) + 1) * (BY + 2 * (nu + 1) + 1) * sizeof(T);
}

// One BX x BY tile of pass A: tile column bx, tile row by; pidx is the tile's slot in a.partial.
// KS: points per thread and round of the staging (0: stage_k's choice). VIN_READY: the caller has
// already written v's window (BX + 2H + 1 square from (x0 - H, y0 - H), zero outside the grid)
// into the first buffer (pass_a_vin), so only f is loaded.
template <typename T, int BX, int BY, int NT, bool NS, int KS = 0, bool VIN_READY = false>
__device__ __forceinline__ void pass_a_tile(const PassAArgs<T>& a, int bx, int by, int pidx,
                                            unsigned char* smem_raw) {
  static_assert(BX % 2 == 0 && BY % 2 == 0, "tiles start on even fine indices");
  const int H = a.nu + 1;
  const int W = BX + 2 * H + 1, Hh = BY + 2 * H + 1;
  T* s0 = reinterpret_cast<T*>(smem_raw);
  T* s1 = s0 + W * Hh;
  T* fs = s1 + W * Hh;
  const int n = a.n;
  const int x0 = bx * BX, y0 = by * BY;
  const int gx0 = x0 - H, gy0 = y0 - H;
  StencilOp<T, NS> op;
  op.load(a.coef, a.level);

  // local (lx, ly) <-> global (gx0 + lx, gy0 + ly)
  if constexpr (VIN_READY) {
    stage_region<NT, KS ? KS : stage_k<BX, BY, NT>()>(
        W, Hh,
        [&](int lx, int ly) {
          const int gx = gx0 + lx, gy = gy0 + ly;
          return inside(gx, gy, n) ? a.f[(size_t)gy * a.ldf + gx] : T(0);
        },
        [&](int lx, int ly, T x) { fs[ly * W + lx] = x; });
  } else {
    stage_region<NT, KS ? KS : stage_k<BX, BY, NT>()>(
        W, Hh,
        [&](int lx, int ly) {
          const int gx = gx0 + lx, gy = gy0 + ly;
          const bool in = inside(gx, gy, n);
          return TwoVals<T>{(in && a.vin) ? a.vin[(size_t)gy * a.ldvin + gx] : T(0),
                            in ? a.f[(size_t)gy * a.ldf + gx] : T(0)};
        },
        [&](int lx, int ly, const TwoVals<T>& x) {
          const int k = ly * W + lx;
          s0[k] = x.a;
          fs[k] = x.b;
        });
  }
  __syncthreads();

  T* src = s0;
  T* dst = s1;
  double ss = 0.0;  // squared residuals of vin on the tile (with a.partial)
  for (int s = 1; s <= a.nu; ++s) {
    const int g = a.nu - s + 1;  // sweep s is needed on the tile grown by g
    const int lo = H - g, R = BX + 2 * g + 1, Ry = BY + 2 * g + 1;
    // from a zero start the first sweep is v = w f, which is what the update gives on zeros
    // (fma(w, f, 0) and every further fma(b, 0, t) = t), in one operation instead of ten
    const bool from_zero = s == 1 && a.vin == nullptr;
    if (s == 1 && a.partial && !from_zero) {
      // the same update as v + w r with the residual r = f - A v explicit, whose squares over the
      // tile's own points give the stopping test of the previous cycle
      for_region<NT>(R, Ry, [&](int rx, int ry) {
        const int lx = lo + rx, ly = lo + ry, k = ly * W + lx;
        T val = T(0);
        if (inside(gx0 + lx, gy0 + ly, n)) {
          const T r = op.res(src, k, W, fs[k]);
          val = fma(op.w(), r, src[k]);
          if ((unsigned)(lx - H) < (unsigned)BX && (unsigned)(ly - H) < (unsigned)BY) ss = fma((double)r, (double)r, ss);
        }
        dst[k] = val;
      });
    } else {
      for_region<NT>(R, Ry, [&](int rx, int ry) {
        const int lx = lo + rx, ly = lo + ry, k = ly * W + lx;
        dst[k] = inside(gx0 + lx, gy0 + ly, n)
                     ? (from_zero ? op.w() * fs[k] : op.jac(src, k, W, fs[k]))
                     : T(0);
      });
    }
    __syncthreads();
    T* t = src; src = dst; dst = t;
  }
  if (a.partial) {
    __shared__ double red[NT / 32];
    const double tot = block_sum<NT>(ss, red);
    if (threadIdx.x == 0) a.partial[pidx] = tot;
  }

  // relaxed v on the tile
  for_region<NT>(BX, BY, [&](int tx, int ty) {
    const int gx = x0 + tx, gy = y0 + ty;
    if (a.vout && inside(gx, gy, n)) a.vout[(size_t)gy * a.ldvout + gx] = src[(ty + H) * W + tx + H];
  });
  // residual on the tile plus one column/row beyond it (full weighting reads it)
  for_region<NT>(BX + 1, BY + 1, [&](int tx, int ty) {
    const int lx = H + tx, ly = H + ty, k = ly * W + lx;
    dst[k] = inside(gx0 + lx, gy0 + ly, n) ? op.res(src, k, W, fs[k]) : T(0);
  });
  __syncthreads();
  // coarse point (I, J) sits on fine (2I+1, 2J+1); this tile owns I in [x0/2, x0/2 + BX/2)
  const int nc = (n - 1) / 2;
  for_region<NT>(BX / 2, BY / 2, [&](int ci, int cj) {
    const int I = x0 / 2 + ci, J = y0 / 2 + cj;
    if (I < nc && J < nc) {
      const int k = (2 * cj + 1 + H) * W + (2 * ci + 1 + H);
      a.fc[(size_t)J * a.ldc + I] = full_weight(dst, k, W);
    }
  });
}

template <typename T, int BX, int BY, int NT, bool NS = false>
__global__ void __launch_bounds__(NT) pass_a_kernel(const PassAArgs<T> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_a_tile<T, BX, BY, NT, NS>(a, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------------
// Pass B: v <- v + P v_c, relax nu times (Algorithm 3, steps 7-8); optionally partial sums of
// ||f - A v||^2 over the tile (one double per block) for the stopping test.
// ---------------------------------------------------------------------------------------------
template <typename T>
struct PassBArgs {
  const T* vin;   // v before correction
  T* vout;        // corrected and relaxed v (must not alias vin)
  const T* f;
  const T* vc;    // coarse-level correction, (n-1)/2 square
  const T* coef;
  const int* skip;
  double* partial;  // nullable: per-block sum of squared residuals of the result
  int ldvin, ldvout, ldf, ldc;
  int n, nu, level;
};

template <typename T, int BX, int BY>
__host__ __device__ constexpr size_t pass_b_smem(int nu, bool norm) {
  // block-sum scratch + two v buffers + f, (BX+2H) x (BY+2H) with H = nu + norm; coarse tile
  return 64 * sizeof(double) +
         size_t(3) * (BX + 2 * (nu + (norm ? 1 : 0))) * (BY + 2 * (nu + (norm ? 1 : 0))) * sizeof(T) +
         size_t(BX / 2 + nu + (norm ? 1 : 0) + 3) * (BY / 2 + nu + (norm ? 1 : 0) + 3) * sizeof(T);
}

// Pass B over the BX x BY points from (x0, y0) (pidx: the slot in a.partial). PB_CS_READY: the
// caller has already written the coarse window into this call's staging buffer (pass_b_cs);
// PB_TO_SMEM: the results go to out_s (pitch out_ld, zero outside the grid) instead of a.vout.
constexpr int PB_CS_READY = 1, PB_TO_SMEM = 2;

// This call's coarse staging buffer in its shared memory (BX x BY points, halo H).
template <typename T, int BX, int BY>
__device__ __forceinline__ T* pass_b_cs(unsigned char* smem_raw, int H) {
  return reinterpret_cast<T*>(smem_raw + 64 * sizeof(double)) + 3 * (BX + 2 * H) * (BY + 2 * H);
}

template <typename T, int BX, int BY, int NT, bool NS, int KS = 0, int MODE = 0>
__device__ __forceinline__ void pass_b_core(const PassBArgs<T>& a, int x0, int y0, int pidx,
                                            unsigned char* smem_raw, T* out_s = nullptr, int out_ld = 0) {
  const int E = a.partial ? 1 : 0;
  const int H = a.nu + E;
  const int W = BX + 2 * H, Hh = BY + 2 * H;
  const int n = a.n, nc = (n - 1) / 2;
  const int gx0 = x0 - H, gy0 = y0 - H;
  // coarse indices that bilinear interpolation reads for fine x in [gx0, gx0 + W)
  const int cx0 = (gx0 >> 1) - 1, cy0 = (gy0 >> 1) - 1;
  const int CW = ((gx0 + W - 1) >> 1) - cx0 + 1, CH = ((gy0 + Hh - 1) >> 1) - cy0 + 1;
  double* red = reinterpret_cast<double*>(smem_raw);  // NT/32 doubles for block_sum
  T* s0 = reinterpret_cast<T*>(smem_raw + 64 * sizeof(double));
  T* s1 = s0 + W * Hh;
  T* fs = s1 + W * Hh;
  T* cs = fs + W * Hh;
  StencilOp<T, NS> op;
  op.load(a.coef, a.level);

  constexpr int K = KS ? KS : stage_k<BX, BY, NT>();
  auto stage_coarse = [&]() {
    if (MODE & PB_CS_READY) return;
    stage_region<NT, K>(
        CW, CH,
        [&](int lx, int ly) {
          const int cx = cx0 + lx, cy = cy0 + ly;
          return inside(cx, cy, nc) ? a.vc[(size_t)cy * a.ldc + cx] : T(0);
        },
        [&](int lx, int ly, T x) { cs[ly * CW + lx] = x; });
  };
  auto cv = [&](int cx, int cy) { return cs[(cy - cy0) * CW + (cx - cx0)]; };
  // the bilinear interpolation P v_c at fine (gx, gy), from the staged coarse window
  auto interp = [&](int gx, int gy) {
    // fine (gx, gy): odd index = coarse point (gx-1)/2; even index between gx/2-1 and gx/2
    T p;
    const bool xo = gx & 1, yo = gy & 1;
    const int hx = gx >> 1, hy = gy >> 1;
    if (xo && yo) {
      p = cv(hx, hy);
    } else if (yo) {
      p = T(0.5) * (cv(hx - 1, hy) + cv(hx, hy));
    } else if (xo) {
      p = T(0.5) * (cv(hx, hy - 1) + cv(hx, hy));
    } else {
      p = T(0.25) * ((cv(hx - 1, hy - 1) + cv(hx, hy - 1)) + (cv(hx - 1, hy) + cv(hx, hy)));
    }
    return p;
  };
  if (W * Hh <= K * NT) {
    // one round: this thread's loads of v and f are in flight while the coarse window is staged
    const int q = NT / W, r = NT - q * W;
    int ly = threadIdx.x / W, lx = threadIdx.x - ly * W;
    int xs[K], ys[K];
    T vr[K], fr[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      xs[u] = lx;
      ys[u] = ly;
      const int gx = gx0 + lx, gy = gy0 + ly;
      const bool in = ly < Hh && inside(gx, gy, n);
      vr[u] = in ? a.vin[(size_t)gy * a.ldvin + gx] : T(0);
      fr[u] = in ? a.f[(size_t)gy * a.ldf + gx] : T(0);
      lx += r;
      ly += q;
      if (lx >= W) {
        lx -= W;
        ++ly;
      }
    }
    stage_coarse();
    __syncthreads();
#pragma unroll
    for (int u = 0; u < K; ++u) {
      if (ys[u] >= Hh) continue;
      const int gx = gx0 + xs[u], gy = gy0 + ys[u], k = ys[u] * W + xs[u];
      s0[k] = inside(gx, gy, n) ? vr[u] + interp(gx, gy) : T(0);
      fs[k] = fr[u];
    }
  } else {
    stage_coarse();
    __syncthreads();
    stage_region<NT, K>(W, Hh, [&](int lx, int ly) {
      const int gx = gx0 + lx, gy = gy0 + ly;
      T v = T(0), fv = T(0);
      if (inside(gx, gy, n)) {
        fv = a.f[(size_t)gy * a.ldf + gx];
        v = a.vin[(size_t)gy * a.ldvin + gx] + interp(gx, gy);
      }
      return TwoVals<T>{v, fv};
    }, [&](int lx, int ly, const TwoVals<T>& x) {
      const int k = ly * W + lx;
      s0[k] = x.a;
      fs[k] = x.b;
    });
  }
  __syncthreads();

  T* src = s0;
  T* dst = s1;
  for (int s = 1; s <= a.nu; ++s) {
    const int g = a.nu - s + E;
    const int lo = H - g, R = BX + 2 * g, Ry = BY + 2 * g;
    for_region<NT>(R, Ry, [&](int rx, int ry) {
      const int lx = lo + rx, ly = lo + ry, k = ly * W + lx;
      dst[k] = inside(gx0 + lx, gy0 + ly, n) ? op.jac(src, k, W, fs[k]) : T(0);
    });
    __syncthreads();
    T* t = src; src = dst; dst = t;
  }
  double ss = 0.0;
  for_region<NT>(BX, BY, [&](int tx, int ty) {
    const int gx = x0 + tx, gy = y0 + ty;
    const int k = (ty + H) * W + tx + H;
    if (MODE & PB_TO_SMEM) {
      out_s[ty * out_ld + tx] = inside(gx, gy, n) ? src[k] : T(0);
    } else if (inside(gx, gy, n)) {
      a.vout[(size_t)gy * a.ldvout + gx] = src[k];
      if (E) {
        const double r = (double)op.res(src, k, W, fs[k]);
        ss = fma(r, r, ss);
      }
    }
  });
  if (E) {
    const double tot = block_sum<NT>(ss, red);
    if (threadIdx.x == 0) a.partial[pidx] = tot;
  }
}

// One BX x BY tile of pass B (tile column bx, row by; pidx: the tile's slot in a.partial).
template <typename T, int BX, int BY, int NT, bool NS, int KS = 0>
__device__ __forceinline__ void pass_b_tile(const PassBArgs<T>& a, int bx, int by, int pidx,
                                            unsigned char* smem_raw) {
  pass_b_core<T, BX, BY, NT, NS, KS>(a, bx * BX, by * BY, pidx, smem_raw);
}

template <typename T, int BX, int BY, int NT, bool NS = false>
__global__ void __launch_bounds__(NT) pass_b_kernel(const PassBArgs<T> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_b_tile<T, BX, BY, NT, NS>(a, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------------
// Zebra line relaxation tables (the kernels are in lines.cuh): per level and direction the Thomas
// factors mm, cp of the line operator and the chunk products pi, rho of the chunked solve.
// ---------------------------------------------------------------------------------------------
// Chunk length of the line solves of a level of side n: the largest power of two <= 16 whose
// 32-lane segment still fits in the line.
__host__ __device__ inline int line_chunk(int n) {
  int mc = 16;
  while (mc > 1 && 32 * mc > n + 1) mc >>= 1;
  return mc;
}

// Offset of the tables of (level l, direction dir) in the table array: per level 2 directions x 4
// tables (mm, cp, pi, rho) of n_l entries; n_l = 2^(k-l) - 1.
// Under semi-coarsening (semi != 0) every level keeps the 2^k - 1 columns, so every table has that
// length.
__host__ __device__ inline size_t line_tab_offset(int k, int l, int dir, int semi = 0) {
  if (semi) return (size_t(2) * l + dir) * 4 * ((size_t(1) << k) - 1);
  size_t off = 0;
  for (int q = 0; q < l; ++q) off += size_t(8) * ((1 << (k - q)) - 1);
  return off + size_t(dir) * 4 * ((1 << (k - l)) - 1);
}

__host__ __device__ inline size_t line_tab_size(int k, int levels, int semi = 0) {
  return line_tab_offset(k, levels, 0, semi);
}

// Dense inverses of the line operators of the levels with side <= LINV_MAX, per level and
// direction n*n entries (row-major, FP64): the FP64 coarse kernel applies them as one short
// matrix-vector product per point instead of the two dependent Thomas sweeps.
constexpr int LINV_MAX = 15;
__host__ __device__ inline size_t line_inv_offset(int k, int l, int dir) {
  size_t off = 0;
  for (int q = 0; q < l; ++q) {
    const size_t m = (size_t(1) << (k - q)) - 1;
    if (m <= LINV_MAX) off += 2 * m * m;
  }
  const size_t n = (size_t(1) << (k - l)) - 1;
  return off + size_t(dir) * n * n;
}

// ---------------------------------------------------------------------------------------------
// Coarse levels: one CTA walks Algorithm 3 for levels lc..L-1 entirely in shared memory.
// ---------------------------------------------------------------------------------------------
template <typename T>
struct CoarseArgs {
  T* v;            // global v at level lc (read when the first call is not zero-start; written back)
  const T* f;      // global f at level lc
  const T* coef;   // coefficient table of all levels (precision T)
  const double* coef64;  // FP64 coefficient table: the coarsest solve is always FP64
  const double* cinv;    // FP64 dense inverse of the coarsest operator when its grid is larger than 1x1
  const int* skip;
  int ldv, ldf;
  int n_lc;        // grid side of level lc
  int lc, L;       // first coarse level and number of levels
  int nu1, nu2;
  int k1, k2;      // counters of the (up to) two calls made at level lc; k2 = 0: one call
  int zero1;       // first call starts from zero
  int adjoint;     // adjoint cycle: nu1 <-> nu2 and the kappa-1 call first
  const T* ltab;   // zebra line tables (precision T); nullptr: damped Jacobi
  const double* linv;  // dense line inverses of the levels with side <= LINV_MAX (FP64 cycles) or nullptr
  int k;           // finest side 2^k - 1 (locates the line tables of a level)
  int xonly;       // zebra relaxations all along x (no alternation)
  // Condensed calls: a call at relative level dcond with counter c is the affine map
  // v <- M_c v + N_c f (S = side^2 unknowns), precomputed from this kernel's own recursion;
  // cmap holds, per class c = 1..ncls (counters >= ncls use the last), M_c then N_c, each stored
  // by columns (entry (k, b) at b * S + k). nullptr: no condensation.
  const T* cmap;
  int dcond, ncls;
  int map_smem;    // copy the maps into shared memory (after the levels) at the start of the walk
  // basis != 0: map mode. basis = 1: block b runs one call of counter k1 at the top level from
  // v = e_b (b < S) or f = e_(b-S); basis = 2: block b runs the calls k1, k2 from v = 0 with
  // f = e_b. Each block writes its result to cmap_out + b * S.
  int basis;
  T* cmap_out;
};

__host__ __device__ inline int coarse_side(int n_lc, int d) {
  int s = n_lc;
  for (int i = 0; i < d; ++i) s = (s - 1) / 2;
  return s;
}

// Jacobi update written as a shallow tree (depth 4 instead of 6) for the latency-bound coarse
// levels: two more FP64 operations per point, more independent work per thread.
template <typename T>
__device__ __forceinline__ T jacobi_update_tree(const Nb<T>& nb, T fv, const Coef<T>& c) {
  const T t1 = fma(c.w, fv, c.b0 * nb.c);
  const T t2 = fma(c.bns, nb.ns, c.bwe * nb.we);
  const T t3 = fma(c.bne, nb.d2, c.bnw * nb.d1);
  return (t1 + t2) + t3;
}

// Shared memory of the coarse kernel: per level two v buffers and f, each (side+2)^2 with a zero
// border, plus one temporary of the largest level; then the zebra line tables of its levels (mm
// and cp per direction, precision T) and the dense line inverses (FP64) of the sides <= LINV_MAX.
__host__ __device__ inline size_t coarse_line_tables(int n_lc, int nlev) {
  size_t tot = 0;
  for (int d = 0; d < nlev; ++d) tot += 4 * size_t(coarse_side(n_lc, d));
  return tot;
}
__host__ __device__ inline size_t coarse_line_inverses(int n_lc, int nlev) {
  size_t tot = 0;
  for (int d = 0; d < nlev; ++d) {
    const size_t s = coarse_side(n_lc, d);
    if (s <= LINV_MAX) tot += 2 * s * s;
  }
  return tot;
}
template <typename T>
__host__ __device__ inline size_t coarse_smem(int n_lc, int nlev) {
  size_t tot = 0;
  for (int d = 0; d < nlev; ++d) {
    const int s = coarse_side(n_lc, d) + 2;
    tot += 3 * size_t(s) * s;
  }
  tot += size_t(n_lc + 2) * (n_lc + 2);
  tot += coarse_line_tables(n_lc, nlev);
  tot = (tot * sizeof(T) + 15) / 16 * 16;
  return tot + coarse_line_inverses(n_lc, nlev) * sizeof(double);
}

// The coarse-level walk, run by one CTA (block index blockIdx.x only in map mode) on the dynamic
// shared memory at smem_raw.
// Shared memory for the condensed-call maps (ncls classes of M and N, S = 49 unknowns each), placed
// after coarse_smem's regions.
template <typename T>
__host__ __device__ inline size_t coarse_map_smem(int ncls) {
  return size_t(ncls) * 2 * 49 * 49 * sizeof(T);
}

// Padded position ((side + 2)^2 buffer with a zero border) of interior point k of a level of the
// given side; magic = ceil(2^32 / side), so that k / side == umulhi(k, magic) for k < 4096.
__device__ __forceinline__ int pad_pos(int k, int side, unsigned magic) {
  const int j = (int)__umulhi((unsigned)k, magic);
  return (j + 1) * (side + 2) + (k - j * side) + 1;
}

template <typename T, int NT, bool LINES, bool NS>
__device__ __forceinline__ void coarse_body(const CoarseArgs<T>& a, unsigned char* smem_raw) {
  static_assert(!(LINES && NS), "line relaxation is for the symmetric operators");
  __shared__ StencilOp<T, NS> cf[MAXL];
  __shared__ int g_side[MAXL], g_off[MAXL + 1], g_magic[MAXL];
  const int nlev = a.L - a.lc;
  T* base = reinterpret_cast<T*>(smem_raw);
  if (threadIdx.x < nlev) cf[threadIdx.x].load(a.coef, a.lc + threadIdx.x);
  if (threadIdx.x == 0) {
    int off = 0;
    for (int d = 0; d < nlev; ++d) {
      const int sd = coarse_side(a.n_lc, d);
      g_side[d] = sd;
      g_off[d] = off;  // v0 at off, v1 at off + P^2, f at off + 2 P^2
      g_magic[d] = (int)((0x100000000ull + sd - 1) / sd);  // k / sd == umulhi(k, magic) for k < 4096
      off += 3 * (sd + 2) * (sd + 2);
    }
    g_off[nlev] = off;
  }
  __syncthreads();
  T* tmp = base + g_off[nlev];
  // zebra tables: level d's mm/cp of direction dir at ltab_s + 4 * (sum of the sides above) + 2 * dir * s
  T* ltab_s = tmp + (a.n_lc + 2) * (a.n_lc + 2);
  double* linv_s = reinterpret_cast<double*>(
      smem_raw + ((size_t)(ltab_s + coarse_line_tables(a.n_lc, nlev) - base) * sizeof(T) + 15) / 16 * 16);
  if (LINES) {
    size_t o = 0, oi = 0;
    for (int d = 0; d < nlev; ++d) {
      const int s = g_side[d];
      for (int dir = 0; dir < 2; ++dir) {
        const T* src = a.ltab + line_tab_offset(a.k, a.lc + d, dir);
        for (int e = threadIdx.x; e < 2 * s; e += NT) ltab_s[o + e] = src[e];
        o += 2 * s;
        if (a.linv && s <= LINV_MAX) {
          const double* isrc = a.linv + line_inv_offset(a.k, a.lc + d, dir);
          for (int e = threadIdx.x; e < s * s; e += NT) linv_s[oi + e] = isrc[e];
          oi += (size_t)s * s;
        }
      }
    }
  }
  // Only the zero borders of the v buffers are ever read before being written (f, the temporary
  // and v interiors are written first), so only those are cleared.
  for (int d = 0; d < nlev; ++d) {
    const int P = g_side[d] + 2;
    T* v0 = base + g_off[d];
    T* v1 = v0 + P * P;
    for (int e = threadIdx.x; e < 4 * (P - 1); e += NT) {
      const int side = e / (P - 1), t = e - side * (P - 1);
      const int k = side == 0 ? t : (side == 1 ? (P - 1) * P + t + 1 : (side == 2 ? (t + 1) * P : t * P + P - 1));
      v0[k] = T(0);
      v1[k] = T(0);
    }
  }
  // condensed-call maps: from shared memory when the launch provides room for them
  const T* cmap = a.cmap;
  if (a.cmap && a.map_smem && !a.basis) {
    T* ms = reinterpret_cast<T*>(smem_raw + coarse_smem<T>(a.n_lc, nlev));
    const int tot = a.ncls * 2 * 49 * 49;
    for (int e = threadIdx.x; e < tot; e += NT) ms[e] = a.cmap[e];
    cmap = ms;
  }
  __syncthreads();

  unsigned cur = 0;  // bit d: which of the two v buffers of level d holds the current iterate
  auto vbuf = [&](int d, int which) { const int P = g_side[d] + 2; return base + g_off[d] + which * P * P; };
  auto fbuf = [&](int d) { const int P = g_side[d] + 2; return base + g_off[d] + 2 * P * P; };
  auto vcur = [&](int d) { return vbuf(d, (cur >> d) & 1u); };
  auto pos = [&](int d, int k) {  // padded position of interior point k of level d
    const int s = g_side[d];
    const int j = (int)__umulhi((unsigned)k, (unsigned)g_magic[d]);
    return (j + 1) * (s + 2) + (k - j * s) + 1;
  };
  {
    const int s = a.n_lc;
    T* fv = fbuf(0);
    T* vv = vbuf(0, 0);
    if (a.basis) {
      const int S = s * s, b = blockIdx.x;
      const int bv = a.basis == 2 ? -1 : b, bf = a.basis == 2 ? b : b - S;
      for (int k = threadIdx.x; k < S; k += NT) {
        vv[pos(0, k)] = (k == bv) ? T(1) : T(0);
        fv[pos(0, k)] = (k == bf) ? T(1) : T(0);
      }
    } else {
      for (int k = threadIdx.x; k < s * s; k += NT) {
        const int j = (int)__umulhi((unsigned)k, (unsigned)g_magic[0]), i = k - j * s;
        fv[pos(0, k)] = a.f[(size_t)j * a.ldf + i];
        if (!a.zero1) vv[pos(0, k)] = a.v[(size_t)j * a.ldv + i];
      }
    }
  }
  __syncthreads();

  const int nu_pre = a.adjoint ? a.nu2 : a.nu1;
  const int nu_post = a.adjoint ? a.nu1 : a.nu2;

  // `sweeps` damped-Jacobi sweeps on level d, ping-ponging between its two v buffers; a zero
  // start makes the first sweep v = w f (the update of v = 0)
  auto relax = [&](int d, int sweeps, bool zero) {
    // level geometry and stencil in registers: the sweeps store to shared memory, which would
    // otherwise make every point reload them
    const int s = g_side[d], P = s + 2;
    const unsigned mg = g_magic[d];
    const T* f = fbuf(d);
    const StencilOp<T, NS> op = cf[d];
    if (zero && sweeps == 0) {
      T* v = vcur(d);
      for (int k = threadIdx.x; k < s * s; k += NT) v[pad_pos(k, s, mg)] = T(0);
      __syncthreads();
      return;
    }
    for (int it = 0; it < sweeps; ++it) {
      const unsigned b = (cur >> d) & 1u;
      const T* src = vbuf(d, b);
      T* dst = vbuf(d, b ^ 1u);
      const bool from_zero = zero && it == 0;
      for (int k = threadIdx.x; k < s * s; k += NT) {
        const int kk = pad_pos(k, s, mg);
        if constexpr (NS) {
          dst[kk] = from_zero ? op.w() * f[kk] : op.jac(src, kk, P, f[kk]);
        } else {
          dst[kk] = from_zero ? op.c.w * f[kk] : jacobi_update_tree(neighbours(src, kk, P), f[kk], op.c);
        }
      }
      cur ^= 1u << d;
      __syncthreads();
    }
  };
  // `sweeps` alternating zebra relaxations on level d, in place: the k-th along x (rows) for even
  // k, along y (columns) for odd k; colour 0 lines then colour 1 lines, one thread per line
  // running the Thomas recurrences with the level's tabulated factors
  auto relax_lines = [&](int d, int sweeps, bool zero) {
    if constexpr (!NS) {
    const int s = g_side[d], P = s + 2;
    T* v = vcur(d);
    const T* f = fbuf(d);
    const Coef<T> c = cf[d].c;
    if (zero) {
      for (int k = threadIdx.x; k < s * s; k += NT) v[pos(d, k)] = T(0);
      __syncthreads();
    }
    size_t o = 0, oi = 0;  // this level's tables in shared memory
    for (int q = 0; q < d; ++q) {
      o += 4 * (size_t)g_side[q];
      if (a.linv && g_side[q] <= LINV_MAX) oi += 2 * (size_t)g_side[q] * g_side[q];
    }
    const bool dense = a.linv && s <= LINV_MAX;
    for (int it = 0; it < sweeps; ++it) {
      const int dir = a.xonly ? 0 : (it & 1);
      const T* mm = ltab_s + o + 2 * dir * s;
      const T* cp = mm + s;
      const double* inv = linv_s + oi + (size_t)dir * s * s;
      const T cl = dir == 0 ? c.cns : c.cwe;
      const int pstep = dir == 0 ? 1 : P, lstep = dir == 0 ? P : 1;
      for (int colour = 0; colour < 2; ++colour) {
        if (dense) {
          // r of every point of this colour's lines into tmp (line-major), then x = T^-1 r
          const int nl = (s - colour + 1) / 2;
          for (int e = threadIdx.x; e < nl * s; e += NT) {
            const int li = e / s, t = e - li * s, L = colour + 2 * li;
            const T* x = v + (L + 1) * lstep + (t + 1) * pstep;
            T r = f[(L + 1) * lstep + (t + 1) * pstep];
            r = fma(-cl, x[-lstep] + x[lstep], r);
            r = fma(-c.cnw, x[-lstep + pstep] + x[lstep - pstep], r);
            r = fma(-c.cne, x[-lstep - pstep] + x[lstep + pstep], r);
            tmp[e] = r;
          }
          __syncthreads();
          for (int e = threadIdx.x; e < nl * s; e += NT) {
            const int li = e / s, t = e - li * s, L = colour + 2 * li;
            const T* r = tmp + li * s;
            const double* row = inv + (size_t)t * s;
            double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
            int q = 0;
            for (; q + 2 < s; q += 3) {
              acc0 = fma(row[q], (double)r[q], acc0);
              acc1 = fma(row[q + 1], (double)r[q + 1], acc1);
              acc2 = fma(row[q + 2], (double)r[q + 2], acc2);
            }
            for (; q < s; ++q) acc0 = fma(row[q], (double)r[q], acc0);
            v[(L + 1) * lstep + (t + 1) * pstep] = (T)((acc0 + acc1) + acc2);
          }
          __syncthreads();
          continue;
        }
        for (int L = colour + 2 * (int)threadIdx.x; L < s; L += 2 * NT) {
          T* x = v + (L + 1) * lstep + pstep;  // point 0 of line L; borders of the buffer are zero
          const T* fl = f + (L + 1) * lstep + pstep;
          const T* Pl = x - lstep;
          const T* Ql = x + lstep;
          T y = T(0);
          for (int t = 0; t < s; ++t) {
            const int o = t * pstep;
            T r = fl[o];
            r = fma(-cl, Pl[o] + Ql[o], r);
            r = fma(-c.cnw, Pl[o + pstep] + Ql[o - pstep], r);
            r = fma(-c.cne, Pl[o - pstep] + Ql[o + pstep], r);
            y = fma(-cp[t], y, mm[t] * r);
            x[o] = y;
          }
          T z = T(0);
          for (int t = s - 1; t >= 0; --t) {
            z = fma(-cp[t], z, x[t * pstep]);
            x[t * pstep] = z;
          }
        }
        __syncthreads();
      }
    }
    }
  };
  auto smooth = [&](int d, int sweeps, bool zero) {
    if constexpr (LINES) relax_lines(d, sweeps, zero); else relax(d, sweeps, zero);
  };
  // f_{d+1} = R (f_d - A v_d)
  auto restrict_residual = [&](int d) {
    const int s = g_side[d], P = s + 2;
    const T* v = vcur(d);
    const T* f = fbuf(d);
    const StencilOp<T, NS> op = cf[d];
    const unsigned mg = g_magic[d];
    for (int k = threadIdx.x; k < s * s; k += NT) {
      const int kk = pad_pos(k, s, mg);
      tmp[kk] = op.res(v, kk, P, f[kk]);
    }
    __syncthreads();
    const int sc = g_side[d + 1];
    const unsigned mgc = g_magic[d + 1];
    T* fc = fbuf(d + 1);
    for (int k = threadIdx.x; k < sc * sc; k += NT) {
      const int J = (int)__umulhi((unsigned)k, mgc), I = k - J * sc;
      // coarse (I, J) sits on fine (2I+1, 2J+1), padded position (2J+2, 2I+2)
      fc[(J + 1) * (sc + 2) + I + 1] = full_weight(tmp, (2 * J + 2) * P + (2 * I + 2), P);
    }
    __syncthreads();
  };
  // v_d += P v_{d+1}; the padded coarse index of coarse (I, J) is (J+1)*Pc + I+1
  auto prolong_add = [&](int d) {
    const int s = g_side[d], Pc = g_side[d + 1] + 2;
    const unsigned mg = g_magic[d];
    T* v = vcur(d);
    const T* vc = vcur(d + 1);
    for (int k = threadIdx.x; k < s * s; k += NT) {
      const int j = (int)__umulhi((unsigned)k, mg), i = k - j * s;
      const int hx = i >> 1, hy = j >> 1;
      T p;
      const bool xo = i & 1, yo = j & 1;
      if (xo && yo) {
        p = vc[(hy + 1) * Pc + hx + 1];
      } else if (yo) {
        p = T(0.5) * (vc[(hy + 1) * Pc + hx] + vc[(hy + 1) * Pc + hx + 1]);
      } else if (xo) {
        p = T(0.5) * (vc[hy * Pc + hx + 1] + vc[(hy + 1) * Pc + hx + 1]);
      } else {
        p = T(0.25) * ((vc[hy * Pc + hx] + vc[hy * Pc + hx + 1]) + (vc[(hy + 1) * Pc + hx] + vc[(hy + 1) * Pc + hx + 1]));
      }
      v[(j + 1) * (s + 2) + i + 1] += p;
    }
    __syncthreads();
  };
  // exact coarsest solve in FP64 whatever T is: division for 1x1, dense inverse otherwise (into the
// other buffer)
  auto coarsest = [&]() {
    const int d = nlev - 1, s = g_side[d];
    const T* f = fbuf(d);
    const unsigned b = (cur >> d) & 1u;
    T* dst = vbuf(d, b ^ 1u);
    if (s == 1) {  // padded 3x3, interior at 4
      if (threadIdx.x == 0) dst[4] = (T)((double)f[4] / a.coef64[(a.L - 1) * NCOEF + C_C0]);
    } else {
      const int N = s * s;
      const unsigned mg = g_magic[d];
      for (int r = threadIdx.x; r < N; r += NT) {
        double acc = 0.0;
        for (int q = 0; q < N; ++q) acc = fma(a.cinv[(size_t)r * N + q], (double)f[pad_pos(q, s, mg)], acc);
        dst[pad_pos(r, s, mg)] = (T)acc;
      }
    }
    cur ^= 1u << d;
    __syncthreads();
  };

  struct Frame { int d, k, state, zero; };
  Frame st[MAXL];
  const int ncalls = a.k2 > 0 ? 2 : 1;
  for (int call = 0; call < ncalls; ++call) {
    int sp = 0;
    st[sp++] = Frame{0, call == 0 ? a.k1 : a.k2, 0, call == 0 ? a.zero1 : 0};
    while (sp > 0) {
      Frame& fr = st[sp - 1];
      if (fr.d == nlev - 1) {  // coarsest level: exact solve (ignores the incoming v)
        coarsest();
        --sp;
        continue;
      }
      if (cmap && fr.d == a.dcond) {  // condensed call: v <- M_c v + N_c f in one pass
        const int d = fr.d, s = g_side[d], S = s * s;
        const unsigned mg = g_magic[d];
        const int cls = (fr.k < a.ncls ? fr.k : a.ncls) - 1;
        const T* Mt = cmap + (size_t)cls * 2 * S * S;
        const T* Nt = Mt + (size_t)S * S;
        const unsigned bsel = (cur >> d) & 1u;
        const T* vsrc = vbuf(d, bsel);
        T* dst = vbuf(d, bsel ^ 1u);
        const T* f = fbuf(d);
        // four threads per output row (aligned lane groups), each taking every fourth column
        for (int base = 0; base < 4 * S; base += NT) {
          const int tid = base + (int)threadIdx.x, k = tid >> 2, p = tid & 3;
          T acc0 = T(0), acc1 = T(0);
          if (k < S) {
            if (!fr.zero)
              for (int b = p; b < S; b += 4) acc0 = fma(Mt[(size_t)b * S + k], vsrc[pad_pos(b, s, mg)], acc0);
            for (int b = p; b < S; b += 4) acc1 = fma(Nt[(size_t)b * S + k], f[pad_pos(b, s, mg)], acc1);
          }
          T acc = acc0 + acc1;
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          acc += __shfl_xor_sync(0xffffffffu, acc, 2);
          if (k < S && p == 0) dst[pad_pos(k, s, mg)] = acc;
        }
        cur ^= 1u << d;
        __syncthreads();
        --sp;
        continue;
      }
      if (fr.state == 0) {
        smooth(fr.d, nu_pre, fr.zero != 0);
        restrict_residual(fr.d);
        fr.state = 1;
        const int kf = a.adjoint ? (fr.k > 1 ? fr.k - 1 : fr.k) : fr.k;
        st[sp++] = Frame{fr.d + 1, kf, 0, 1};
        continue;
      }
      if (fr.state == 1) {
        fr.state = 2;
        const int ks = a.adjoint ? (fr.k > 1 ? fr.k : 0) : (fr.k > 1 ? fr.k - 1 : 0);
        if (ks > 0) {
          st[sp++] = Frame{fr.d + 1, ks, 0, 0};
          continue;
        }
      }
      prolong_add(fr.d);
      smooth(fr.d, nu_post, false);
      --sp;
    }
  }
  {
    const int s = a.n_lc;
    const T* vv = vcur(0);
    if (a.basis) {
      T* out = a.cmap_out + (size_t)blockIdx.x * s * s;
      for (int k = threadIdx.x; k < s * s; k += NT) out[k] = vv[pos(0, k)];
    } else {
      for (int k = threadIdx.x; k < s * s; k += NT) {
        const int j = (int)__umulhi((unsigned)k, (unsigned)g_magic[0]), i = k - j * s;
        a.v[(size_t)j * a.ldv + i] = vv[pos(0, k)];
      }
    }
  }
}

template <typename T, int NT, bool LINES, bool NS = false>
__global__ void __launch_bounds__(NT) coarse_kernel(const CoarseArgs<T> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  coarse_body<T, NT, LINES, NS>(a, smem_raw);
}

// ---------------------------------------------------------------------------------------------
// Condensed child calls. The two calls that a call at level lc-1 makes at level lc (counters k and
// k-1, the first from v = 0, Algorithm 3) together with everything below them are one linear map of
// the restricted residual: v_lc = P_c f_lc, c = min(k, levels - lc + 1) (a call's subtree depends on
// its counter only up to the number of levels below it). P_c is computed once per handle by the
// FP64 coarse kernel in map mode (f = e_b, basis = 2) and stored row by row (pitch pld, rows padded
// with zeros to 16 bytes) in the cycle's precision. Applying it is one matrix-vector product
// instead of the walk's dozens of barrier-separated phases on one SM; it is the same linear map,
// rounded once per entry and once per dot product instead of along the walk.
//
// One warp per row: lane l accumulates the 16-byte chunks l, l + 32, ... of the row in order, then
// a fixed shuffle tree sums the lanes, so a row's result does not depend on which CTA computes it.
// Rows are dealt to warps round-robin over `parts` CTAs (the fused call's cluster, or the grid of
// children_kernel).
// ---------------------------------------------------------------------------------------------
// Rows of P that part `part` of `parts` computes: a contiguous block [lo(part), lo(part + 1)).
__host__ __device__ inline int child_rows_lo(int S, int part, int parts) { return (int)((long long)S * part / parts); }

// Ask L2 for part `part`'s rows of P ahead of the matrix-vector product (one bulk prefetch by one
// thread; the rows are contiguous and 16-byte aligned, pld being a whole number of 16-byte units).
template <typename T>
__device__ __forceinline__ void children_prefetch(const T* pmap, int pld, int S, int part, int parts) {
  if (threadIdx.x != 0 || pmap == nullptr) return;
  const int lo = child_rows_lo(S, part, parts), hi = child_rows_lo(S, part + 1, parts);
  if (hi <= lo) return;
  const T* p = pmap + (size_t)lo * pld;
  const unsigned bytes = (unsigned)((size_t)(hi - lo) * pld * sizeof(T));
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// RG rows a warp streams at once and CH 16-byte chunks per lane and row issued together. Inside a
// fused call (16 CTAs, many rows per warp): FP64 rows (up to 512 entries here) take one round trip
// for two rows, FP32 rows (up to 1024) two for four rows. A stand-alone launch gives each warp about
// one row and streams it eight chunks per lane at a time.
// STAGED: this part's rows of P were copied to shared memory beforehand (`staged`, row lo first).
template <typename T, int NT, int RG = (sizeof(T) == 8 ? 2 : 4), int CH = 4, bool STAGED = false>
__device__ __forceinline__ void children_matvec(const T* __restrict__ pmap, int pld, const CoarseArgs<T>& a,
                                                int part, int parts, T* fs, const T* staged = nullptr) {
  const int s = a.n_lc, S = s * s;
  // f of level lc into shared memory (four loads per thread in flight), zero padding up to pld
  stage_region<NT, 4>(
      s, s, [&](int i, int j) { return a.f[(size_t)j * a.ldf + i]; },
      [&](int i, int j, T x) { fs[j * s + i] = x; });
  for (int b = S + (int)threadIdx.x; b < pld; b += NT) fs[b] = T(0);
  __syncthreads();
  constexpr int NW = NT / 32;
  constexpr int VW = 16 / sizeof(T);  // elements per 16-byte chunk
  const int lane = threadIdx.x & 31, stride = NW;
  const int lo = child_rows_lo(S, part, parts), hi = child_rows_lo(S, part + 1, parts);
  for (int k0 = lo + (threadIdx.x >> 5); k0 < hi; k0 += RG * stride) {
    T acc[RG];
    const T* row[RG];
#pragma unroll
    for (int g = 0; g < RG; ++g) {
      acc[g] = T(0);
      const int k = k0 + g * stride;
      if constexpr (STAGED) row[g] = staged + (size_t)((k < hi ? k : k0) - lo) * pld;
      else row[g] = pmap + (size_t)(k < hi ? k : k0) * pld;
    }
#pragma unroll CH
    for (int b = VW * lane; b < pld; b += 32 * VW) {
      if constexpr (VW == 4) {
        const float4 x = *reinterpret_cast<const float4*>(fs + b);
        float4 q[RG];
#pragma unroll
        for (int g = 0; g < RG; ++g) q[g] = *reinterpret_cast<const float4*>(row[g] + b);
#pragma unroll
        for (int g = 0; g < RG; ++g) {
          acc[g] = fma(q[g].x, x.x, acc[g]);
          acc[g] = fma(q[g].y, x.y, acc[g]);
          acc[g] = fma(q[g].z, x.z, acc[g]);
          acc[g] = fma(q[g].w, x.w, acc[g]);
        }
      } else {
        const double2 x = *reinterpret_cast<const double2*>(fs + b);
        double2 q[RG];
#pragma unroll
        for (int g = 0; g < RG; ++g) q[g] = *reinterpret_cast<const double2*>(row[g] + b);
#pragma unroll
        for (int g = 0; g < RG; ++g) {
          acc[g] = fma(q[g].x, x.x, acc[g]);
          acc[g] = fma(q[g].y, x.y, acc[g]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < RG; ++g) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], o);
      const int k = k0 + g * stride;
      if (lane == 0 && k < hi) {
        const int j = k / s, i = k - j * s;
        a.v[(size_t)j * a.ldv + i] = acc[g];
      }
    }
  }
}

constexpr int CHILD_PARTS = 16;  // the fused call's cluster size, and the fewest CTAs of children_kernel

// The condensed child calls as their own launch (calls not fused with their parent's passes), one
// row per warp where the grid allows.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) children_kernel(const T* __restrict__ pmap, int pld, const CoarseArgs<T> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  children_matvec<T, NT, 1, 8>(pmap, pld, a, blockIdx.x, gridDim.x, reinterpret_cast<T*>(smem_raw));
}

// Column-major FP64 maps (entry (k, b) at b * S + k, as map mode writes them) to row-major maps in
// T with row pitch pld and zero padding.
template <typename T>
__global__ void pmap_convert_kernel(const double* __restrict__ src, int S, int pld, T* __restrict__ dst) {
  const size_t tot = (size_t)S * pld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / pld), b = (int)(e - (size_t)k * pld);
    dst[e] = b < S ? (T)src[(size_t)b * S + k] : T(0);
  }
}

// ---------------------------------------------------------------------------------------------
// One call at the level just above the coarse kernel's, in one launch: a cluster with one CTA per
// TILE x TILE tile of that level runs pass A, then its CTA of rank 0 walks the coarse calls below
// it (the coarse kernel's work), then the cluster runs pass B. The two hand-offs go through global
// memory (the relaxed v and coarse f of pass A, the coarse v of the walk) between cluster barriers,
// whose release/acquire order makes those writes visible to every CTA of the cluster. Replaces the
// three launches pass A, coarse kernel, pass B of that call with one; every point's arithmetic is
// the same, so results equal the three-launch form bit for bit. Launched with a cluster of
// ceil(n / TILE)^2 CTAs (at most 16, the non-portable cluster size).
// ---------------------------------------------------------------------------------------------
constexpr int CALL_MAX_CTAS = 16;

template <typename T, int TILE>
__host__ __device__ constexpr size_t call_cluster_smem_tiles(int nu1, int nu2) {
  return pass_a_smem<T, TILE, TILE>(nu1) > pass_b_smem<T, TILE, TILE>(nu2, false)
             ? pass_a_smem<T, TILE, TILE>(nu1)
             : pass_b_smem<T, TILE, TILE>(nu2, false);
}

template <typename T, int NT, int TILE, bool NS = false>
__global__ void __launch_bounds__(NT)
    call_cluster_kernel(const PassAArgs<T> pa, const CoarseArgs<T> ca, const PassBArgs<T> pb, const T* pmap,
                        int pld) {
  if (pa.skip && *pa.skip) return;  // the same flag for every CTA: the whole cluster returns
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
  const int rank = (int)cluster.block_rank(), size = (int)cluster.num_blocks();
  const int tx = (pa.n + TILE - 1) / TILE, ntiles = tx * tx;
  children_prefetch(pmap, pld, ca.n_lc * ca.n_lc, rank, size);  // lands in L2 while pass A runs
  for (int t = rank; t < ntiles; t += size) {
    pass_a_tile<T, TILE, TILE, NT, NS>(pa, t % tx, t / tx, 0, smem_raw);
    __syncthreads();  // the next tile reuses the shared memory
  }
  cluster.sync();
  if (pmap) {  // the child calls condensed: every CTA computes its share of v_lc = P_c f_lc
    children_matvec<T, NT>(pmap, pld, ca, rank, size, reinterpret_cast<T*>(smem_raw));
  } else if (rank == 0) {
    coarse_body<T, NT, false, NS>(ca, smem_raw);
  }
  cluster.sync();
  for (int t = rank; t < ntiles; t += size) {
    pass_b_tile<T, TILE, TILE, NT, NS>(pb, t % tx, t / tx, 0, smem_raw);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// One call two levels above the coarse kernel's, in one cluster launch: pass A at level l, then its
// one or two child calls at level l+1 -- each pass A at l+1, the condensed grandchildren
// v_{l+2} = P_c f_{l+2} (children_matvec), pass B at l+1 -- then pass B at level l (Algorithm 3 with
// the recursion unrolled two levels deep). Every hand-off goes through global memory between
// cluster barriers; every point's arithmetic is that of the separate launches, so the results equal
// them bit for bit. Launched with a cluster of CALL_MAX_CTAS CTAs; tiles TILE1 at level l, TILE2 at
// level l+1.
// ---------------------------------------------------------------------------------------------
template <typename T>
struct Call2Args {
  PassAArgs<T> pa1;        // level l
  PassBArgs<T> pb1;
  PassAArgs<T> pa2[2];     // level l+1: first child (from zero), second child (from its v)
  PassBArgs<T> pb2;
  CoarseArgs<T> cc;        // v, f and side of level l+2 for the condensed grandchildren
  const T* pmap[2];        // P of the first and second child's counter class
  int pld;
  int children;            // 1 or 2
};

template <typename T, int TILE1, int TILE2>
__host__ __device__ constexpr size_t call2_smem(int nu1, int nu2) {
  return call_cluster_smem_tiles<T, TILE1>(nu1, nu2) > call_cluster_smem_tiles<T, TILE2>(nu1, nu2)
             ? call_cluster_smem_tiles<T, TILE1>(nu1, nu2)
             : call_cluster_smem_tiles<T, TILE2>(nu1, nu2);
}

template <typename T, int NT, int TILE1, int TILE2>
__global__ void __launch_bounds__(NT) call2_cluster_kernel(const Call2Args<T> a) {
  if (a.pa1.skip && *a.pa1.skip) return;  // the same flag for every CTA: the whole cluster returns
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
  const int rank = (int)cluster.block_rank(), size = (int)cluster.num_blocks();
  const int tx1 = (a.pa1.n + TILE1 - 1) / TILE1, nt1 = tx1 * tx1;
  const int tx2 = (a.pb2.n + TILE2 - 1) / TILE2, nt2 = tx2 * tx2;
  children_prefetch(a.pmap[0], a.pld, a.cc.n_lc * a.cc.n_lc, rank, size);
  if (a.children > 1) children_prefetch(a.pmap[1], a.pld, a.cc.n_lc * a.cc.n_lc, rank, size);
  for (int t = rank; t < nt1; t += size) {
    pass_a_tile<T, TILE1, TILE1, NT, false>(a.pa1, t % tx1, t / tx1, 0, smem_raw);
    __syncthreads();
  }
  cluster.sync();
  for (int c = 0; c < a.children; ++c) {
    for (int t = rank; t < nt2; t += size) {
      pass_a_tile<T, TILE2, TILE2, NT, false>(a.pa2[c], t % tx2, t / tx2, 0, smem_raw);
      __syncthreads();
    }
    cluster.sync();
    children_matvec<T, NT>(a.pmap[c], a.pld, a.cc, rank, size, reinterpret_cast<T*>(smem_raw));
    cluster.sync();
    for (int t = rank; t < nt2; t += size) {
      pass_b_tile<T, TILE2, TILE2, NT, false>(a.pb2, t % tx2, t / tx2, 0, smem_raw);
      __syncthreads();
    }
    cluster.sync();
  }
  for (int t = rank; t < nt1; t += size) {
    pass_b_tile<T, TILE1, TILE1, NT, false>(a.pb1, t % tx1, t / tx1, 0, smem_raw);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Setup: fine stencil (Section 4), Galerkin coarse stencils A^{l+1} = R A^l P, coefficient
// tables in double and float, stencil derivatives, and the dense inverse of the coarsest operator.
// ---------------------------------------------------------------------------------------------
__device__ inline double hat1(int d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); }

__device__ inline void fill_coef(const double st[9], double omega, double* out, float* out32) {
  const double c0 = st[4];
  const double w = omega / c0;
  double c[NCOEF];
  for (int q = 0; q < NCOEF; ++q) c[q] = 0.0;
  c[C_C0] = c0;
  c[C_WE] = st[3];  // west (dy=0, dx=-1); east st[5] equal by symmetry
  c[C_NS] = st[1];  // south (dy=-1, dx=0); north st[7]
  c[C_NW] = st[6];  // north-west (dy=+1, dx=-1); south-east st[2]
  c[C_NE] = st[8];  // north-east (dy=+1, dx=+1); south-west st[0]
  c[C_W] = w;
  c[C_B0] = 1.0 - w * c0;
  c[C_BWE] = -w * c[C_WE];
  c[C_BNS] = -w * c[C_NS];
  c[C_BNW] = -w * c[C_NW];
  c[C_BNE] = -w * c[C_NE];
  for (int q = 0; q < 9; ++q) c[C_ST + q] = st[q];
  for (int q = 0; q < NCOEF; ++q) {
    out[q] = c[q];
    out32[q] = (float)c[q];
  }
}

// ---- double-double arithmetic (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2): a value hi + lo with
// |lo| <= ulp(hi)/2, about 106 significant bits. Used only at setup, to round results once.
struct DD {
  double hi, lo;
};
__device__ inline DD dd_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return DD{s, e};
}
__device__ inline DD dd_fast_two_sum(double a, double b) {  // requires |a| >= |b|
  const double s = __dadd_rn(a, b);
  return DD{s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ inline DD dd_two_prod(double a, double b) {  // exact product via a fused multiply-add
  const double p = __dmul_rn(a, b);
  return DD{p, __fma_rn(a, b, -p)};
}
__device__ inline DD dd_add(DD a, DD b) {
  DD s = dd_two_sum(a.hi, b.hi);
  const DD t = dd_two_sum(a.lo, b.lo);
  s = dd_fast_two_sum(s.hi, __dadd_rn(s.lo, t.hi));
  return dd_fast_two_sum(s.hi, __dadd_rn(s.lo, t.lo));
}
__device__ inline DD dd_mul(DD a, DD b) {
  const DD p = dd_two_prod(a.hi, b.hi);
  return dd_fast_two_sum(p.hi, __dadd_rn(p.lo, __fma_rn(a.hi, b.lo, __dmul_rn(a.lo, b.hi))));
}
__device__ inline DD dd_div_small_int(DD a, double m) {  // a / m for a small positive integer m
  const double q1 = __ddiv_rn(a.hi, m);
  const DD p = dd_two_prod(q1, m);
  const double r = __dadd_rn(__dsub_rn(__dsub_rn(a.hi, p.hi), p.lo), a.lo);
  return dd_fast_two_sum(q1, __ddiv_rn(r, m));
}
__device__ inline DD dd_neg(DD a) { return DD{-a.hi, -a.lo}; }

// cos(theta), sin(theta) correctly rounded to double (up to arguments within ~1e-30 of a rounding
// boundary): Cody-Waite reduction by pi/2 = P1 + P2 + P3 (the binary expansion of pi/2 split into
// three doubles), then the Taylor series of cos and sin on |r| <= pi/4 in double-double, rounded
// once. Valid for |theta| <= 1e4.
__device__ inline void dd_cos_sin(double theta, double* c_out, double* s_out) {
  const double P1 = 0x1.921fb54442d18p+0, P2 = 0x1.1a62633145c07p-54, P3 = -0x1.f1976b7ed8fbcp-110;
  const double kd = rint(__ddiv_rn(theta, P1));
  DD r{theta, 0.0};
  r = dd_add(r, dd_neg(dd_two_prod(kd, P1)));
  r = dd_add(r, dd_neg(dd_two_prod(kd, P2)));
  r = dd_add(r, dd_neg(dd_two_prod(kd, P3)));
  const DD r2 = dd_mul(r, r);
  DD cs{1.0, 0.0}, sn = r, tc{1.0, 0.0}, ts = r;
  for (int m = 1; m <= 16; ++m) {  // terms r^(2m)/(2m)! and r^(2m+1)/(2m+1)!
    tc = dd_div_small_int(dd_div_small_int(dd_mul(tc, r2), 2.0 * m - 1.0), 2.0 * m);
    ts = dd_div_small_int(dd_div_small_int(dd_mul(ts, r2), 2.0 * m), 2.0 * m + 1.0);
    cs = dd_add(cs, (m & 1) ? dd_neg(tc) : tc);
    sn = dd_add(sn, (m & 1) ? dd_neg(ts) : ts);
  }
  const int q = ((int)fmod(kd, 4.0) + 4) & 3;
  DD c, s;
  if (q == 0) { c = cs; s = sn; }
  else if (q == 1) { c = dd_neg(sn); s = cs; }
  else if (q == 2) { c = dd_neg(cs); s = dd_neg(sn); }
  else { c = sn; s = dd_neg(cs); }
  *c_out = __dadd_rn(c.hi, c.lo);
  *s_out = __dadd_rn(s.hi, s.lo);
}

// One thread builds all stencils; st index (dy+1)*3 + (dx+1).
// Every stencil is rounded from an exactly known value, so any correctly rounding evaluation
// gives the same bits: the fine entries are evaluated in a fixed order of correctly rounded
// operations (no contraction into fused multiply-adds) from correctly rounded cos and sin; each
// Galerkin entry is a sum of exact products (the transfer weights are powers of two) accumulated
// in double-double and rounded once; the coarse centre follows from the zero-row-sum identity.
// Section 4 stencil on an m x m grid (h = 1/(m+1)) from correctly rounded C, S, as a fixed sequence
// of correctly rounded operations.
__device__ inline void section4_stencil(double C, double S, double eps, int m, double st[9]) {
  const double h = __ddiv_rn(1.0, (double)(m + 1));
  const double h2 = __dmul_rn(h, h);
  const double cross = __dmul_rn(__dmul_rn(__dmul_rn(0.5, __dsub_rn(1.0, eps)), C), S);  // ((0.5(1-eps))C)S
  const double we = -__dadd_rn(__dmul_rn(C, C), __dmul_rn(__dmul_rn(eps, S), S));       // -(CC + (eps S)S)
  const double ns = -__dadd_rn(__dmul_rn(__dmul_rn(eps, C), C), __dmul_rn(S, S));       // -((eps C)C + SS)
  st[4] = __dmul_rn(2.0, __dadd_rn(1.0, eps));
  st[3] = st[5] = we;
  st[1] = st[7] = ns;
  st[6] = cross;   // NW
  st[2] = cross;   // SE
  st[8] = -cross;  // NE
  st[0] = -cross;  // SW
  for (int q = 0; q < 9; ++q) st[q] = __ddiv_rn(st[q], h2);
}

// rediscretized != 0: coarse stencils are the Section 4 stencil on each coarse grid instead of
// the Galerkin products.
// First-order upwind convection b . grad u added to a stencil of grid side m (1/h = m + 1), the
// same rounded operations as the oracle: cx = |bx| (m+1), cy = |by| (m+1), centre += (cx + cy),
// and the upwind neighbour (west for bx > 0, east for bx < 0; south / north for by) -= cx (cy).
__device__ inline void add_convection(double bx, double by, int m, double st[9]) {
  const double cx = __dmul_rn(fabs(bx), (double)(m + 1));
  const double cy = __dmul_rn(fabs(by), (double)(m + 1));
  st[4] = __dadd_rn(st[4], __dadd_rn(cx, cy));
  if (bx > 0.0) st[3] = __dsub_rn(st[3], cx);
  else if (bx < 0.0) st[5] = __dsub_rn(st[5], cx);
  if (by > 0.0) st[1] = __dsub_rn(st[1], cy);
  else if (by < 0.0) st[7] = __dsub_rn(st[7], cy);
}

__global__ void setup_stencils_kernel(double theta, double eps, int n, int levels, double omega,
                                      double* coef, float* coef32, double* stencils, double* dstencil,
                                      int rediscretized, int semi = 0, double bx = 0.0, double by = 0.0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double h = __ddiv_rn(1.0, (double)(n + 1));
  const double h2 = __dmul_rn(h, h);
  double C, S;
  dd_cos_sin(theta, &C, &S);
  double st[9];
  section4_stencil(C, S, eps, n, st);
  if (bx != 0.0 || by != 0.0) add_convection(bx, by, n, st);
  // derivatives of the Section 4 entries with respect to theta and eps, scaled by 1/h^2
  {
    const double s2 = sin(2.0 * theta), c2 = cos(2.0 * theta);
    double* dt = dstencil;
    double* de = dstencil + 9;
    dt[4] = 0.0;
    dt[3] = dt[5] = (1.0 - eps) * s2;
    dt[1] = dt[7] = -(1.0 - eps) * s2;
    dt[6] = dt[2] = 0.5 * (1.0 - eps) * c2;
    dt[8] = dt[0] = -0.5 * (1.0 - eps) * c2;
    de[4] = 2.0;
    de[3] = de[5] = -S * S;
    de[1] = de[7] = -C * C;
    de[6] = de[2] = -0.5 * C * S;
    de[8] = de[0] = 0.5 * C * S;
    for (int q = 0; q < 18; ++q) dstencil[q] /= h2;
  }
  for (int l = 0; l < levels; ++l) {
    for (int q = 0; q < 9; ++q) stencils[l * 9 + q] = st[q];
    fill_coef(st, omega, coef + l * NCOEF, coef32 + l * NCOEF);
    // A_c(D) = sum_{a,b} r(a) S(b) p(a + b - 2D) with r = p/4, p the bilinear hat (separable):
    // (A P e_J)(y) = sum_b S(b) p(y + b - 2J) and (R g)(I) = sum_a r(a) g(2I + a).
    // Semi-coarsening along y: the x factors are the identity (r_x = p_x = delta, no halving), and
    // r_y = p_y / 2. Every product is the entry times a power of two, so the sum is exact.
    double sc[9];
    for (int Dy = -1; Dy <= 1; ++Dy)
      for (int Dx = -1; Dx <= 1; ++Dx) {
        DD acc{0.0, 0.0};
        for (int ay = -1; ay <= 1; ++ay)
          for (int ax = -1; ax <= 1; ++ax) {
            const double r = semi ? (ax == 0 ? 0.5 * hat1(ay) : 0.0) : 0.25 * hat1(ay) * hat1(ax);
            if (r == 0.0) continue;
            for (int by = -1; by <= 1; ++by)
              for (int bx = -1; bx <= 1; ++bx) {
                const double px = semi ? (ax + bx == Dx ? 1.0 : 0.0) : hat1(ax + bx - 2 * Dx);
                const double pv = hat1(ay + by - 2 * Dy) * px;
                if (pv != 0.0) acc = dd_add(acc, DD{__dmul_rn(__dmul_rn(r, st[(by + 1) * 3 + (bx + 1)]), pv), 0.0});
              }
          }
        sc[(Dy + 1) * 3 + (Dx + 1)] = __dadd_rn(acc.hi, acc.lo);
      }
    // exact coarse stencils sum to zero (the fine stencil annihilates constants and the Galerkin
    // map keeps the entry sum); evaluating the centre from that identity, off-centre entries
    // summed in row-major order, stops FP64 rounding of the sum from growing 4x per level
    double off = 0.0;
    for (int q = 0; q < 9; ++q)
      if (q != 4) off = __dadd_rn(off, sc[q]);
    sc[4] = -off;
    for (int q = 0; q < 9; ++q) st[q] = sc[q];
    if (rediscretized) {
      section4_stencil(C, S, eps, ((n + 1) >> (l + 1)) - 1, st);
      if (bx != 0.0 || by != 0.0) add_convection(bx, by, ((n + 1) >> (l + 1)) - 1, st);
    }
  }
}

// Dense inverse of the coarsest operator (N = s*s <= 225) by Gauss-Jordan elimination without
// pivoting (the matrix is symmetric positive definite). One block; work[N*N] is scratch.
__global__ void coarsest_inverse_kernel(const double* stencils, int level, int s, double* work, double* inv,
                                        float* inv32) {
  const int N = s * s;
  const double* st = stencils + level * 9;
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) {
    const int r = k / N, q = k - r * N;
    const int jr = r / s, ir = r - jr * s, jq = q / s, iq = q - jq * s;
    const int dy = jq - jr, dx = iq - ir;
    double v = 0.0;
    if (dy >= -1 && dy <= 1 && dx >= -1 && dx <= 1) v = st[(dy + 1) * 3 + (dx + 1)];
    work[k] = v;
    inv[k] = (r == q) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ double piv;
  for (int p = 0; p < N; ++p) {
    if (threadIdx.x == 0) piv = work[p * N + p];
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      work[p * N + q] *= ip;
      inv[p * N + q] *= ip;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N * N; k += blockDim.x) {
      const int r = k / N, q = k - r * N;
      if (r != p) {
        const double m = work[r * N + p];
        if (q != p) work[k] -= m * work[p * N + q];
        inv[k] -= m * inv[p * N + q];
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x)
      if (r != p) work[r * N + p] = 0.0;
    __syncthreads();
  }
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) inv32[k] = (float)inv[k];
}

// ---------------------------------------------------------------------------------------------
// Whole-grid helpers (one point per thread): apply / residual with partial sums, dot products,
// vector updates for PCG, finalisation of reductions.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Nb<T> neighbours_global(const T* v, int i, int j, int n, int ld) {
  auto at = [&](int ii, int jj) { return inside(ii, jj, n) ? v[(size_t)jj * ld + ii] : T(0); };
  Nb<T> nb;
  nb.c = v[(size_t)j * ld + i];
  nb.we = at(i - 1, j) + at(i + 1, j);
  nb.ns = at(i, j - 1) + at(i, j + 1);
  nb.d1 = at(i - 1, j + 1) + at(i + 1, j - 1);
  nb.d2 = at(i + 1, j + 1) + at(i - 1, j - 1);
  return nb;
}

// out = A v (f == nullptr) or out = f - A v; partial sums of out^2 when partial != nullptr.
template <typename T, int NT, bool NS = false>
__global__ void __launch_bounds__(NT) apply_kernel(const T* __restrict__ v, const T* __restrict__ f, T* out,
                                                   const T* coef, int level, int n, int ld, double* partial,
                                                   const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[NT / 32];
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  double ss = 0.0;
  if constexpr (NS) {
    StencilOp<T, true> op;
    op.load(coef, level);
    if (i < n && j < n) {
      T s9[9];  // the 3x3 neighbourhood, zero outside the grid; centre at index 4, row stride 3
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const int ii = i + q % 3 - 1, jj = j + q / 3 - 1;
        s9[q] = inside(ii, jj, n) ? v[(size_t)jj * ld + ii] : T(0);
      }
      const T r = f ? op.res(s9, 4, 3, f[(size_t)j * ld + i]) : op.app(s9, 4, 3);
      if (out) out[(size_t)j * ld + i] = r;
      ss = (double)r * (double)r;
    }
  } else {
    const Coef<T> c = load_coef(coef, level);
    if (i < n && j < n) {
      const Nb<T> nb = neighbours_global(v, i, j, n, ld);
      const T r = f ? residual_at(nb, f[(size_t)j * ld + i], c) : apply_at(nb, c);
      if (out) out[(size_t)j * ld + i] = r;
      ss = (double)r * (double)r;
    }
  }
  if (partial) {
    const double t = block_sum<NT>(ss, red);
    if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// q = A p with partial sums of p.q (PCG).
template <int NT>
__global__ void __launch_bounds__(NT) apply_dot_kernel(const double* __restrict__ p, double* q, const double* coef,
                                                       int n, double* partial, const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[NT / 32];
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  const Coef<double> c = load_coef(coef, 0);
  double ss = 0.0;
  if (i < n && j < n) {
    const Nb<double> nb = neighbours_global(p, i, j, n, n);
    const double r = apply_at(nb, c);
    q[(size_t)j * n + i] = r;
    ss = nb.c * r;
  }
  const double t = block_sum<NT>(ss, red);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// partial sums of x.y (and of x.z into partial2 when z != nullptr) over a flat array of len
template <int NT>
__global__ void __launch_bounds__(NT) dot_kernel(const double* x, const double* y, const double* z, size_t len,
                                                 double* partial, double* partial2, const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[NT / 32];
  double s1 = 0.0, s2 = 0.0;
  for (size_t k = blockIdx.x * (size_t)NT + threadIdx.x; k < len; k += (size_t)gridDim.x * NT) {
    s1 = fma(x[k], y[k], s1);
    if (z) s2 = fma(x[k], z[k], s2);
  }
  double t = block_sum<NT>(s1, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
  if (z) {
    __syncthreads();
    t = block_sum<NT>(s2, red);
    if (threadIdx.x == 0) partial2[blockIdx.x] = t;
  }
}

// Deterministic sum of np partials (fixed order), valid in thread 0.
template <int NT>
__device__ __forceinline__ double sum_partials(const double* partial, int np, double* red) {
  double s = 0.0;
  for (int k = threadIdx.x; k < np; k += NT) s += partial[k];
  return block_sum<NT>(s, red);
}

// Scalar slots of the solver state on the device.
enum {
  S_FNORM2 = 0,   // ||f||^2 (or ||b||^2)
  S_RZ,           // r.z of the previous PCG iteration
  S_ALPHA,
  S_BETA,
  S_TOL,
  S_LAST,         // last relative residual
  NSCAL = 8
};
// Integer slots
// I_ERR: set by a kernel whose bounded wait ran out; I_BAR, I_BAR + 1: the persistent deep calls'
// grid barrier (arrivals, generation)
enum { I_DONE = 0, I_COUNT, I_MAX, I_ERR, I_BAR, NINT = 6 };

template <int NT>
__global__ void __launch_bounds__(NT) sum_to_scalar_kernel(const double* partial, int np, double* out) {
  __shared__ double red[NT / 32];
  const double s = sum_partials<NT>(partial, np, red);
  if (threadIdx.x == 0) *out = s;
}

// After a cycle (or a PCG update): rho = sqrt(sum) / ||f||; record it; decide whether to go on.
// cond: conditional-node handle of the enclosing WHILE loop (used when use_cond != 0).
template <int NT>
__global__ void __launch_bounds__(NT) finish_step_kernel(const double* partial, int np, double* scal, int* ints,
                                                         double* hist, cudaGraphConditionalHandle cond,
                                                         int use_cond, int pre = 0) {
  __shared__ double red[NT / 32];
  if (ints[I_DONE]) {
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double s = sum_partials<NT>(partial, np, red);
  if (pre && threadIdx.x == 0) {
    // the norm is that of the iterate before this cycle (formed by its first sweep): after
    // k = ints[I_COUNT] completed cycles. Stop before the cycle (the rest of it is skipped)
    // once k >= 1 cycles reached tol, or k reached the limit; otherwise count the cycle.
    const double fn = sqrt(scal[S_FNORM2]);
    const double rho = fn > 0.0 ? sqrt(s) / fn : sqrt(s);
    const int k = ints[I_COUNT];
    if (k >= 1) {
      hist[k - 1] = rho;
      scal[S_LAST] = rho;
    }
    const bool stop = k >= 1 && ((rho <= scal[S_TOL]) || (k >= ints[I_MAX]));
    if (stop) ints[I_DONE] = 1;
    else ints[I_COUNT] = k + 1;
    if (use_cond) cudaGraphSetConditional(cond, stop ? 0 : 1);
    return;
  }
  if (threadIdx.x == 0) {
    const double fn = sqrt(scal[S_FNORM2]);
    const double rho = fn > 0.0 ? sqrt(s) / fn : sqrt(s);
    const int k = ints[I_COUNT];
    hist[k] = rho;
    ints[I_COUNT] = k + 1;
    scal[S_LAST] = rho;
    const bool stop = (rho <= scal[S_TOL]) || (k + 1 >= ints[I_MAX]);
    if (stop) ints[I_DONE] = 1;
    if (use_cond) cudaGraphSetConditional(cond, stop ? 0 : 1);
  }
}

// PCG: alpha = rz / (p.q) from the p.q partials.
template <int NT>
__global__ void __launch_bounds__(NT) pcg_alpha_kernel(const double* partial, int np, double* scal, const int* ints) {
  __shared__ double red[NT / 32];
  if (ints[I_DONE]) return;
  const double pq = sum_partials<NT>(partial, np, red);
  if (threadIdx.x == 0) scal[S_ALPHA] = scal[S_RZ] / pq;
}

// PCG: beta = (r.z_new [- r.z_old]) / rz_old; rz <- r.z_new.
template <int NT>
__global__ void __launch_bounds__(NT) pcg_beta_kernel(const double* partial, const double* partial2, int np,
                                                      int flexible, double* scal, const int* ints) {
  __shared__ double red[NT / 32];
  if (ints[I_DONE]) return;
  const double rz_new = sum_partials<NT>(partial, np, red);
  __syncthreads();
  double rz_old_new = 0.0;
  if (flexible) rz_old_new = sum_partials<NT>(partial2, np, red);
  if (threadIdx.x == 0) {
    scal[S_BETA] = (flexible ? (rz_new - rz_old_new) : rz_new) / scal[S_RZ];
    scal[S_RZ] = rz_new;
  }
}

// x += alpha p; r -= alpha q; partial sums of r.r
template <int NT>
__global__ void __launch_bounds__(NT) pcg_update_kernel(double* x, double* r, const double* p, const double* q,
                                                        size_t len, const double* scal, double* partial,
                                                        const int* ints) {
  if (ints[I_DONE]) return;
  __shared__ double red[NT / 32];
  const double alpha = scal[S_ALPHA];
  double s = 0.0;
  for (size_t k = blockIdx.x * (size_t)NT + threadIdx.x; k < len; k += (size_t)gridDim.x * NT) {
    x[k] = fma(alpha, p[k], x[k]);
    const double rk = fma(-alpha, q[k], r[k]);
    r[k] = rk;
    s = fma(rk, rk, s);
  }
  const double t = block_sum<NT>(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// p = z + beta p (use_beta) or p = z; optional copy z -> zold
template <int NT>
__global__ void __launch_bounds__(NT) pcg_p_kernel(double* p, const double* z, double* zold, size_t len,
                                                   const double* scal, int use_beta, const int* ints) {
  if (ints[I_DONE]) return;
  const double beta = use_beta ? scal[S_BETA] : 0.0;
  for (size_t k = blockIdx.x * (size_t)NT + threadIdx.x; k < len; k += (size_t)gridDim.x * NT) {
    const double zk = z[k];
    p[k] = use_beta ? fma(beta, p[k], zk) : zk;
    if (zold) zold[k] = zk;
  }
}

// x += y (the two halves of the symmetrised preconditioner).
template <int NT>
__global__ void __launch_bounds__(NT) vec_add_kernel(double* x, const double* y, size_t len, const int* skip) {
  if (skip && *skip) return;
  for (size_t k = blockIdx.x * (size_t)NT + threadIdx.x; k < len; k += (size_t)gridDim.x * NT) x[k] += y[k];
}

// Parameter gradients: partial sums of lambda . (dA/dtheta u) and lambda . (dA/deps u).
template <int NT>
__global__ void __launch_bounds__(NT) grad_kernel(const double* lam, const double* u, int n, const double* dst,
                                                  double* partial_th, double* partial_ep) {
  __shared__ double red[NT / 32];
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  double s_th = 0.0, s_ep = 0.0;
  if (i < n && j < n) {
    double a_th = 0.0, a_ep = 0.0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx, jj = j + dy;
        if (inside(ii, jj, n)) {
          const double uv = u[(size_t)jj * n + ii];
          a_th = fma(dst[(dy + 1) * 3 + (dx + 1)], uv, a_th);
          a_ep = fma(dst[9 + (dy + 1) * 3 + (dx + 1)], uv, a_ep);
        }
      }
    const double l = lam[(size_t)j * n + i];
    s_th = l * a_th;
    s_ep = l * a_ep;
  }
  double t = block_sum<NT>(s_th, red);
  if (threadIdx.x == 0) partial_th[blockIdx.y * gridDim.x + blockIdx.x] = t;
  __syncthreads();
  t = block_sum<NT>(s_ep, red);
  if (threadIdx.x == 0) partial_ep[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// ---------------------------------------------------------------------------------------------
// Mixed precision: FP32 cycles inside FP64 iterative refinement.
// ---------------------------------------------------------------------------------------------
// x += d (FP64 += FP32 correction), pointwise; x has pitch n, d pitch ldd
template <int NT>
__global__ void __launch_bounds__(NT) ir_add_kernel(double* x, const float* d, int n, int ldd, const int* skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  if (i < n && j < n) x[(size_t)j * n + i] += (double)d[(size_t)j * ldd + i];
}

// r = f - A x in FP64, stored rounded to FP32 as the right-hand side of the next FP32 cycle, with
// partial sums of r^2 (FP64) for the stopping test
template <int NT>
__global__ void __launch_bounds__(NT) ir_residual_kernel(const double* __restrict__ x, const double* __restrict__ f,
                                                         float* r32, int ldr, const double* coef, int n,
                                                         double* partial, const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[NT / 32];
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  const Coef<double> c = load_coef(coef, 0);
  double ss = 0.0;
  if (i < n && j < n) {
    const double r = residual_at(neighbours_global(x, i, j, n, n), f[(size_t)j * n + i], c);
    r32[(size_t)j * ldr + i] = (float)r;
    ss = r * r;
  }
  const double t = block_sum<NT>(ss, red);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// y = (double) x or y = (float) x, pointwise (mixed-precision preconditioner hand-off)
template <int NT, typename S, typename D>
__global__ void __launch_bounds__(NT) convert_kernel(D* y, int ldy, const S* x, int ldx, int n, const int* skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  if (i < n && j < n) y[(size_t)j * ldy + i] = (D)x[(size_t)j * ldx + i];
}

// Throughput probe of the FP64 pipe: 8 independent chains of dependent fused multiply-adds per
// thread (the result is consumed so the work cannot be removed).
__global__ void fp64_rate_kernel(double* sink, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.678) sink[0] = s;  // never true for these inputs
}

__global__ void reset_state_kernel(int* ints, int max_iters, double* scal, double tol) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ints[I_DONE] = 0;
    ints[I_COUNT] = 0;
    ints[I_MAX] = max_iters;
    scal[S_TOL] = tol;
  }
}

}  // namespace kc
