// Zebra line relaxation (Section 4, solvers 3-4): every line of one colour is solved exactly with
// the neighbouring lines (the other colour) held fixed; colour 0 (lines 0, 2, 4, ...) first, then
// colour 1. A relaxation along x solves rows, one along y solves columns.
//
// The line operator of a level is the constant symmetric tridiagonal matrix tridiag(a, d, a) of the
// level's stencil (d the centre, a the west/east entry for rows, south/north for columns). Its
// Thomas factors are the same for every line, so they are tabulated once per level and direction:
//   mm[t] = 1 / (d - a cp[t-1]),  cp[t] = a mm[t]          (cp[-1] = 0)
// forward:  y[t] = mm[t] r[t] - cp[t] y[t-1];  backward: x[t] = y[t] - cp[t] x[t+1].
//
// Both recurrences are split into chunks of MC points, one chunk per lane. A chunk is solved with a
// zero carry-in, and the carries follow from a warp scan of the chunks' affine maps. The chunk
// products are also tabulated:
//   pi[t]  = prod_{s = chunk start}^{t} (-cp[s])                 (d y[t] / d y[chunk start - 1])
//   rho[t] = prod_{s = t}^{min(chunk end, n) - 1} (-cp[s])       (d x[t] / d x[chunk end])
// A CTA owns R lines of one colour (one warp per line) and walks them in segments of 32 MC points,
// staged in shared memory with coalesced loads. The forward pass goes left to right and stores the
// y values in place, and the backward pass goes right to left; each carries the recurrence across
// segments. The lines' old values are never read (a line solve does not use them), so the
// update is in place.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace kc {

// One thread per (level, direction). Levels with side <= LINV_MAX also get the dense inverse
// (column q solves T x = e_q with the same factors). Under semi-coarsening every line has 2^k - 1
// points.
__global__ void line_tables_kernel(const double* coef, int k, int levels, double* tab, float* tab32,
                                   double* linv, int semi) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * levels) return;
  const int l = id >> 1, dir = id & 1;
  const int n = semi ? (1 << k) - 1 : (1 << (k - l)) - 1, mc = line_chunk(n);
  const double d = coef[l * NCOEF + C_C0];
  const double a = coef[l * NCOEF + (dir == 0 ? C_WE : C_NS)];
  const size_t off = line_tab_offset(k, l, dir, semi);
  double* mm = tab + off;
  double* cp = mm + n;
  double* pi = cp + n;
  double* rho = pi + n;
  double c = 0.0;
  for (int t = 0; t < n; ++t) {
    const double m = 1.0 / (d - a * c);
    c = a * m;
    mm[t] = m;
    cp[t] = c;
    pi[t] = (t % mc == 0) ? -c : pi[t - 1] * -c;
  }
  for (int t = n - 1; t >= 0; --t) {
    const bool last = (t % mc == mc - 1) || t == n - 1;
    rho[t] = last ? -cp[t] : rho[t + 1] * -cp[t];
  }
  for (int q = 0; q < 4 * n; ++q) tab32[off + q] = (float)tab[off + q];
  if (!semi && n <= LINV_MAX) {
    double* inv = linv + line_inv_offset(k, l, dir);
    for (int q = 0; q < n; ++q) {
      double y[LINV_MAX];
      double yp = 0.0;
      for (int t = 0; t < n; ++t) {
        yp = mm[t] * ((t == q ? 1.0 : 0.0) - a * yp);
        y[t] = yp;
      }
      double x = 0.0;
      for (int t = n - 1; t >= 0; --t) {
        x = y[t] - cp[t] * x;
        inv[(size_t)t * n + q] = x;
      }
    }
  }
}

template <typename T>
struct LineArgs {
  T* v;            // level array, updated in place (lines of `colour` only)
  const T* f;
  const T* coef;   // coefficient table (precision T)
  const T* tab;    // mm, cp, pi, rho of this level and direction, n entries each
  const int* skip;
  const T* vc;     // nullable (rows only): neighbouring lines are read as v + P vc, the coarse-grid
                   // correction of Algorithm 3 applied on the fly (pass B folded in)
  int n;           // points per line
  int nl;          // number of lines (n for square grids; the rows of a semi-coarsened level)
  int ld, level, ldc;
  int colour;      // 0: lines 0, 2, ...; 1: lines 1, 3, ...
  int zero;        // neighbouring lines are zero (first relaxation from a zero start)
  int semi;        // vc is a semi-coarsened correction: fine row 2J+1 receives coarse row J
};

// Bilinear prolongation of the coarse correction at fine (gx, gy), in the arithmetic order of
// pass B: coarse point (I, J) sits on fine (2I+1, 2J+1); zero outside the coarse grid.
template <typename T>
__device__ __forceinline__ T prolong_point(const T* vc, int ldc, int nc, int gx, int gy) {
  auto cv = [&](int cx, int cy) { return inside(cx, cy, nc) ? vc[(size_t)cy * ldc + cx] : T(0); };
  const bool xo = gx & 1, yo = gy & 1;
  const int hx = gx >> 1, hy = gy >> 1;
  if (xo && yo) return cv(hx, hy);
  if (yo) return T(0.5) * (cv(hx - 1, hy) + cv(hx, hy));
  if (xo) return T(0.5) * (cv(hx, hy - 1) + cv(hx, hy));
  return T(0.25) * ((cv(hx - 1, hy - 1) + cv(hx, hy - 1)) + (cv(hx - 1, hy) + cv(hx, hy)));
}

// R lines per CTA; MC points per lane and segment chunk.
template <int R, int MC>
struct LineGeom {
  static constexpr int S = 32 * MC;                       // points per segment
  static constexpr int PADN = S + 2 + (S + 2) / MC + 1;  // padded neighbour row (halo of one each side)
  static constexpr int PADS = S + S / MC + 1;             // padded segment row
  // one padding slot per MC points: lane k's j-th point sits at k (MC + 1) + j, so the 32 lanes of
  // a warp hit distinct bank pairs
  __device__ static int pad(int u) { return u + u / MC; }
};

template <typename T, int R, int MC>
__host__ __device__ constexpr size_t line_smem() {
  using G = LineGeom<R, MC>;
  return sizeof(T) * (size_t(R + 1) * G::PADN + size_t(R) * G::PADS + size_t(4) * G::PADS);
}

// Inclusive warp scan of affine maps x -> A x + B, composed from lane 0 upwards (UP) or from lane
// 31 downwards: the result at lane k is F_k o F_(k-1) o ... o F_0 (UP) or F_k o ... o F_31.
template <bool UP, typename T>
__device__ __forceinline__ void affine_scan(T& A, T& B, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T Ao = UP ? __shfl_up_sync(0xffffffffu, A, o) : __shfl_down_sync(0xffffffffu, A, o);
    const T Bo = UP ? __shfl_up_sync(0xffffffffu, B, o) : __shfl_down_sync(0xffffffffu, B, o);
    if (UP ? lane >= o : lane + o < 32) {
      B = fma(A, Bo, B);
      A = A * Ao;
    }
  }
}

// One colour of one zebra relaxation: lines are rows (DIR 0) or columns (DIR 1).
template <typename T, int DIR, int R, int MC>
__global__ void __launch_bounds__(32 * R) line_relax_kernel(const LineArgs<T> a) {
  if (a.skip && *a.skip) return;
  using G = LineGeom<R, MC>;
  constexpr int NT = 32 * R, S = G::S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* nb = reinterpret_cast<T*>(smem_raw);   // (R+1) neighbour lines, points s0-1 .. s0+S
  T* fs = nb + (R + 1) * G::PADN;           // R lines: f, then y, then x of the segment
  T* tb = fs + R * G::PADS;                 // tables mm, cp, pi, rho of the segment
  const int n = a.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t pstr = DIR == 0 ? 1 : (size_t)a.ld;  // step along a line
  const size_t lstr = DIR == 0 ? (size_t)a.ld : 1;  // step between lines
  const int first = a.colour + 2 * R * blockIdx.x;  // line of warp 0; warp r owns first + 2r
  const Coef<T> c = load_coef(a.coef, a.level);
  const T cl = DIR == 0 ? c.cns : c.cwe;  // coupling to the same point of a neighbouring line
  const T* mmg = a.tab;
  const T* cpg = mmg + n;
  const T* pig = cpg + n;
  const T* rhog = pig + n;
  const int nseg = (n + S - 1) / S;
  const int nc = (n - 1) / 2;

  // cooperative loads/stores of a tile of `rows` lines x `len` points; lines `l0 + 2q`; the inner
  // index runs along the line for rows (coalesced) and across lines for columns (stride-2 columns)
  auto tile = [&](int rows, int len, auto fn) {
    for (int e = threadIdx.x; e < rows * len; e += NT) {
      int q, u;
      if (DIR == 0) { q = e / len; u = e - q * len; } else { u = e / rows; q = e - u * rows; }
      fn(q, u);
    }
  };

  // ---------------- forward: y = L^{-1} r, left to right ----------------
  T yseg = T(0);  // y at the last point of the previous segment (this warp's line)
  T yv[MC];       // after the loop: y of this lane's chunk of the last segment (kept for the backward pass)
  for (int sg = 0; sg < nseg; ++sg) {
    const int s0 = sg * S;
    __syncthreads();
    tile(R + 1, S + 2, [&](int q, int u) {
      const int L = first - 1 + 2 * q, t = s0 - 1 + u;
      T val = T(0);
      if (!a.zero && L >= 0 && L < a.nl && t >= 0 && t < n) {
        val = a.v[(size_t)L * lstr + (size_t)t * pstr];
        if (DIR == 0 && a.vc) {
          // colour-0 neighbours are odd rows: under semi-coarsening row 2J+1 takes coarse row J
          val = val + (a.semi ? a.vc[(size_t)(L >> 1) * a.ldc + t] : prolong_point(a.vc, a.ldc, nc, t, L));
        }
      }
      nb[q * G::PADN + G::pad(u)] = val;
    });
    tile(R, S, [&](int q, int u) {
      const int L = first + 2 * q, t = s0 + u;
      fs[q * G::PADS + G::pad(u)] = (L < a.nl && t < n) ? a.f[(size_t)L * lstr + (size_t)t * pstr] : T(0);
    });
    for (int u = threadIdx.x; u < S; u += NT) {
      const int t = s0 + u;
      if (t < n) {
        tb[0 * G::PADS + G::pad(u)] = mmg[t];
        tb[1 * G::PADS + G::pad(u)] = cpg[t];
        tb[2 * G::PADS + G::pad(u)] = pig[t];
      }
    }
    __syncthreads();
    const T* P = nb + warp * G::PADN;
    const T* Q = P + G::PADN;
    T* fy = fs + warp * G::PADS;
    T y = T(0), A = T(1), B = T(0);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const int u = lane * MC + j;
      yv[j] = T(0);
      if (s0 + u < n) {
        // neighbour points t-1, t, t+1 sit at u, u+1, u+2
        const T pm = P[G::pad(u)], p0 = P[G::pad(u + 1)], pp = P[G::pad(u + 2)];
        const T qm = Q[G::pad(u)], q0 = Q[G::pad(u + 1)], qp = Q[G::pad(u + 2)];
        T r = fy[G::pad(u)];
        r = fma(-cl, p0 + q0, r);
        r = fma(-c.cnw, pp + qm, r);
        r = fma(-c.cne, pm + qp, r);
        y = fma(-tb[1 * G::PADS + G::pad(u)], y, tb[0 * G::PADS + G::pad(u)] * r);
        yv[j] = y;
        A = tb[2 * G::PADS + G::pad(u)];
        B = y;
      }
    }
    affine_scan<true>(A, B, lane);
    T Ain = __shfl_up_sync(0xffffffffu, A, 1), Bin = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) { Ain = T(1); Bin = T(0); }
    const T yin = fma(Ain, yseg, Bin);
    yseg = __shfl_sync(0xffffffffu, fma(A, yseg, B), 31);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const int u = lane * MC + j;
      if (s0 + u < n) yv[j] = fma(tb[2 * G::PADS + G::pad(u)], yin, yv[j]);
    }
    if (sg == nseg - 1) break;  // the last segment's y stays in registers
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const int u = lane * MC + j;
      if (s0 + u < n) fy[G::pad(u)] = yv[j];
    }
    __syncthreads();
    tile(R, S, [&](int q, int u) {
      const int L = first + 2 * q, t = s0 + u;
      if (L < a.nl && t < n) a.v[(size_t)L * lstr + (size_t)t * pstr] = fs[q * G::PADS + G::pad(u)];
    });
  }

  // ---------------- backward: x = U^{-1} y, right to left ----------------
  T xseg = T(0);  // x at the first point of the next segment
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s0 = sg * S;
    __syncthreads();
    if (sg < nseg - 1) {
      tile(R, S, [&](int q, int u) {
        const int L = first + 2 * q, t = s0 + u;
        fs[q * G::PADS + G::pad(u)] = (L < a.nl && t < n) ? a.v[(size_t)L * lstr + (size_t)t * pstr] : T(0);
      });
    }
    for (int u = threadIdx.x; u < S; u += NT) {
      const int t = s0 + u;
      if (t < n) {
        tb[1 * G::PADS + G::pad(u)] = cpg[t];
        tb[3 * G::PADS + G::pad(u)] = rhog[t];
      }
    }
    __syncthreads();
    T* fy = fs + warp * G::PADS;
    if (sg < nseg - 1) {
#pragma unroll
      for (int j = 0; j < MC; ++j) yv[j] = fy[G::pad(lane * MC + j)];
    }
    T x = T(0), E = T(1), D = T(0);
#pragma unroll
    for (int j = MC - 1; j >= 0; --j) {
      const int u = lane * MC + j;
      if (s0 + u < n) {
        x = fma(-tb[1 * G::PADS + G::pad(u)], x, yv[j]);
        yv[j] = x;
        E = tb[3 * G::PADS + G::pad(u)];
        D = x;
      }
    }
    affine_scan<false>(E, D, lane);
    T Eup = __shfl_down_sync(0xffffffffu, E, 1), Dup = __shfl_down_sync(0xffffffffu, D, 1);
    if (lane == 31) { Eup = T(1); Dup = T(0); }
    const T xin = fma(Eup, xseg, Dup);
    xseg = __shfl_sync(0xffffffffu, fma(E, xseg, D), 0);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const int u = lane * MC + j;
      if (s0 + u < n) fy[G::pad(u)] = fma(tb[3 * G::PADS + G::pad(u)], xin, yv[j]);
    }
    __syncthreads();
    tile(R, S, [&](int q, int u) {
      const int L = first + 2 * q, t = s0 + u;
      if (L < a.nl && t < n) a.v[(size_t)L * lstr + (size_t)t * pstr] = fs[q * G::PADS + G::pad(u)];
    });
  }
}

// ---------------------------------------------------------------------------------------------
// Long rows, few of them (the deep levels of semi-coarsening keep every column): one row per
// cluster of CL CTAs (CL SMs), so no segments and no single SM's FP64 pipe in the way (one SM
// needs about 15 us for a 4095-point row). Each thread streams its chunk from global memory; the
// chunk products are formed on the fly (two more FP64 operations per point than the tabulated
// ones), so only mm and cp are read. CTA rank r of a cluster owns
// points [r NT MC, (r+1) NT MC) of the cluster's row; the CTA totals of the two scans are
// exchanged through distributed shared memory between cluster barriers.
// ---------------------------------------------------------------------------------------------
// The same scan over the first N lanes only (log2 N steps); lanes >= N are not read.
template <bool UP, int N, typename T>
__device__ __forceinline__ void affine_scan_n(T& A, T& B, int lane) {
#pragma unroll
  for (int o = 1; o < N; o <<= 1) {
    const T Ao = UP ? __shfl_up_sync(0xffffffffu, A, o) : __shfl_down_sync(0xffffffffu, A, o);
    const T Bo = UP ? __shfl_up_sync(0xffffffffu, B, o) : __shfl_down_sync(0xffffffffu, B, o);
    if (UP ? lane >= o : lane + o < N) {
      B = fma(A, Bo, B);
      A = A * Ao;
    }
  }
}

template <typename T, int MC, int NT, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) line_cluster_kernel(const LineArgs<T> a) {
  namespace cg = cooperative_groups;
  if (a.skip && *a.skip) return;  // the flag is the same for every CTA of the grid
  constexpr int NW = NT / 32;
  static_assert(NW <= 32, "one warp scans the warp totals");
  __shared__ T wa[NW], wb[NW];
  __shared__ T ca, cb;  // this CTA's total map, read by the other CTAs of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int n = a.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int L = a.colour + 2 * (blockIdx.x / CL);  // one row per cluster
  const size_t ld = (size_t)a.ld;
  const Coef<T> c = load_coef(a.coef, a.level);
  const T* mmg = a.tab;
  const T* cpg = mmg + n;
  const int t0 = (rank * NT + threadIdx.x) * MC;
  const int cnt = max(0, min(MC, n - t0));
  const bool hasP = !a.zero && L - 1 >= 0, hasQ = !a.zero && L + 1 < a.nl;
  const int nc = (n - 1) / 2;
  auto nbv = [&](bool has, int row, int t) -> T {
    if (!has || t < 0 || t >= n) return T(0);
    T val = a.v[(size_t)row * ld + t];
    if (a.vc) val = val + (a.semi ? a.vc[(size_t)(row >> 1) * a.ldc + t] : prolong_point(a.vc, a.ldc, nc, t, row));
    return val;
  };
  const T* fl = a.f + (size_t)L * ld;

  T bv[MC], gv[MC];
  {
    T pm = nbv(hasP, L - 1, t0 - 1), p0 = nbv(hasP, L - 1, t0);
    T qm = nbv(hasQ, L + 1, t0 - 1), q0 = nbv(hasQ, L + 1, t0);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      bv[j] = T(0);
      gv[j] = T(1);
      if (j < cnt) {
        const int t = t0 + j;
        const T pp = nbv(hasP, L - 1, t + 1), qp = nbv(hasQ, L + 1, t + 1);
        T r = fl[t];
        r = fma(-c.cns, p0 + q0, r);
        r = fma(-c.cnw, pp + qm, r);
        r = fma(-c.cne, pm + qp, r);
        bv[j] = mmg[t] * r;
        gv[j] = -cpg[t];
        pm = p0; p0 = pp; qm = q0; q0 = qp;
      }
    }
  }
  // ---- forward
  T y = T(0), A = T(1);
#pragma unroll
  for (int j = 0; j < MC; ++j) {
    if (j < cnt) {
      y = fma(gv[j], y, bv[j]);
      bv[j] = y;
      A = A * gv[j];
    }
  }
  T B = y;
  affine_scan<true>(A, B, lane);
  if (lane == 31) { wa[warp] = A; wb[warp] = B; }
  __syncthreads();
  if (warp == 0) {
    T a2 = lane < NW ? wa[lane] : T(1), b2 = lane < NW ? wb[lane] : T(0);
    affine_scan_n<true, NW>(a2, b2, lane);
    if (lane < NW) { wa[lane] = a2; wb[lane] = b2; }
    if (lane == NW - 1) { ca = a2; cb = b2; }
  }
  cluster.sync();
  // y entering this CTA's first point: the lower ranks' maps composed in parallel (lane q reads
  // rank q's total) and applied from zero
  T ycta;
  {
    T qa = T(1), qb = T(0);
    if (lane < rank) {
      qa = *cluster.map_shared_rank(&ca, lane);
      qb = *cluster.map_shared_rank(&cb, lane);
    }
    affine_scan_n<true, CL>(qa, qb, lane);
    ycta = __shfl_sync(0xffffffffu, qb, rank > 0 ? rank - 1 : 0);
    if (rank == 0) ycta = T(0);
  }
  T Ain = __shfl_up_sync(0xffffffffu, A, 1), Bin = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) { Ain = T(1); Bin = T(0); }
  const T ywarp = warp > 0 ? fma(wa[warp - 1], ycta, wb[warp - 1]) : ycta;
  const T yin = fma(Ain, ywarp, Bin);
  {
    T pr = T(1);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      if (j < cnt) {
        pr = pr * gv[j];
        bv[j] = fma(pr, yin, bv[j]);
      }
    }
  }
  // ---- backward
  T x = T(0), E = T(1);
#pragma unroll
  for (int j = MC - 1; j >= 0; --j) {
    if (j < cnt) {
      x = fma(gv[j], x, bv[j]);
      bv[j] = x;
      E = E * gv[j];
    }
  }
  T D = x;
  affine_scan<false>(E, D, lane);
  cluster.sync();  // every CTA has read the forward totals (ca, cb, wa, wb)
  if (lane == 0) { wa[warp] = E; wb[warp] = D; }
  __syncthreads();
  if (warp == 0) {
    T a2 = lane < NW ? wa[lane] : T(1), b2 = lane < NW ? wb[lane] : T(0);
    affine_scan_n<false, NW>(a2, b2, lane);
    if (lane < NW) { wa[lane] = a2; wb[lane] = b2; }
    if (lane == 0) { ca = a2; cb = b2; }
  }
  cluster.sync();
  // x at the first point after this CTA: the higher ranks' maps composed in parallel, from zero
  T xcta;
  {
    T qa = T(1), qb = T(0);
    if (lane > rank && lane < CL) {
      qa = *cluster.map_shared_rank(&ca, lane);
      qb = *cluster.map_shared_rank(&cb, lane);
    }
    affine_scan_n<false, CL>(qa, qb, lane);
    xcta = __shfl_sync(0xffffffffu, qb, rank + 1 < CL ? rank + 1 : 0);
    if (rank + 1 >= CL) xcta = T(0);
  }
  T Eup = __shfl_down_sync(0xffffffffu, E, 1), Dup = __shfl_down_sync(0xffffffffu, D, 1);
  if (lane == 31) { Eup = T(1); Dup = T(0); }
  const T xwarp = warp + 1 < NW ? fma(wa[warp + 1], xcta, wb[warp + 1]) : xcta;
  const T xin = fma(Eup, xwarp, Dup);
  T* vl = a.v + (size_t)L * ld;
  T q = T(1);
#pragma unroll
  for (int j = MC - 1; j >= 0; --j) {
    if (j < cnt) {
      q = q * gv[j];
      vl[t0 + j] = fma(q, xin, bv[j]);
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------------------------
// Semi-coarsening along y (Section 4, solvers 5-6): f_c = R_y (f - A v), R_y = (1/4)[1 2 1] across
// rows, and v += P_y v_c (coarse row J on fine row 2J+1, rows 2J averaging J-1 and J). Every level
// keeps the nx columns; rows are ny (fine) and (ny-1)/2 (coarse).
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T residual_rect(const T* v, const T* f, int i, int j, int nx, int ny, int ldv, int ldf,
                                           const Coef<T>& c) {
  auto at = [&](int x, int y) { return ((unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny) ? v[(size_t)y * ldv + x] : T(0); };
  Nb<T> nb;
  nb.c = at(i, j);
  nb.we = at(i - 1, j) + at(i + 1, j);
  nb.ns = at(i, j - 1) + at(i, j + 1);
  nb.d1 = at(i - 1, j + 1) + at(i + 1, j - 1);
  nb.d2 = at(i + 1, j + 1) + at(i - 1, j - 1);
  return residual_at(nb, f[(size_t)j * ldf + i], c);
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) restrict_y_kernel(const T* __restrict__ v, const T* __restrict__ f, T* fc,
                                                       const T* coef, int level, int nx, int nyc, int ldv, int ldf,
                                                       int ldc, int vzero, const int* skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int J = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  if (i >= nx || J >= nyc) return;
  const Coef<T> c = load_coef(coef, level);
  const int ny = 2 * nyc + 1, y = 2 * J + 1;
  T r0, r1, r2;
  if (vzero) {
    r0 = f[(size_t)(y - 1) * ldf + i];
    r1 = f[(size_t)y * ldf + i];
    r2 = f[(size_t)(y + 1) * ldf + i];
  } else {
    r0 = residual_rect(v, f, i, y - 1, nx, ny, ldv, ldf, c);
    r1 = residual_rect(v, f, i, y, nx, ny, ldv, ldf, c);
    r2 = residual_rect(v, f, i, y + 1, nx, ny, ldv, ldf, c);
  }
  fc[(size_t)J * ldc + i] = fma(T(0.25), r2, fma(T(0.5), r1, T(0.25) * r0));
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) prolong_y_add_kernel(T* v, const T* __restrict__ vc, int nx, int nyc, int ldv,
                                                          int ldc, const int* skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
  const int ny = 2 * nyc + 1;
  if (i >= nx || y >= ny) return;
  T p;
  if (y & 1) {
    p = vc[(size_t)(y >> 1) * ldc + i];
  } else {
    const int J = y >> 1;  // between coarse rows J - 1 and J
    const T lo = J >= 1 ? vc[(size_t)(J - 1) * ldc + i] : T(0);
    const T hi = J < nyc ? vc[(size_t)J * ldc + i] : T(0);
    p = T(0.5) * (lo + hi);
  }
  v[(size_t)y * ldv + i] += p;
}

}  // namespace kc
