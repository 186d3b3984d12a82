// FP32 fused level passes for the large levels of the FP32 cycle of the mixed forms: pass B as a
// register pipeline from side 4095, pass A (all large levels) and pass B below 4095 as
// shared-memory tiles (at the end of this file).
//
// FP32 level passes are bound by HBM bandwidth and instruction issue, not by arithmetic: the
// generic shared-memory tile kernels spend their issue slots on index arithmetic and barriers. In
// the register pipeline one warp owns a vertical strip of 128 columns (4 consecutive columns per
// lane, read with float4 loads) and streams down a chunk of rows. Every stage of the pass
// (interpolation, Jacobi sweeps) keeps a window of three rows in registers and gets the
// column to the left and right of its 4 columns from the neighbouring lanes by warp shuffles. No
// shared memory, no barriers; the next input row is loaded while the current one is processed.
// Each stage loses one column per side, so a strip yields 120 output columns; rows of neighbouring
// chunks overlap by a few rows (read again, mostly from L2).
//
// Arrays must be 16-byte aligned with a pitch that is a multiple of 4 floats (coarse arrays:
// multiple of 2); the host falls back to the tile kernels otherwise.
#pragma once
#include "kernels.cuh"

namespace kc {

constexpr int SF_COLS = 120;  // output columns per warp
constexpr int SF_WARPS = 4;   // warps per CTA (independent strips)
constexpr int SF_AHEAD_B = 4; // input rows loaded ahead of use (at 4095^2: 115 -> 107 us against 3)

struct Row6 {  // 4 columns of one row plus the neighbouring column on each side
  float l, v[4], r;
};

__device__ __forceinline__ float r6(const Row6& R, int k) {  // k in -1..4
  return k < 0 ? R.l : (k > 3 ? R.r : R.v[k]);
}

__device__ __forceinline__ Row6 with_halo(const float (&v)[4]) {
  Row6 R;
#pragma unroll
  for (int k = 0; k < 4; ++k) R.v[k] = v[k];
  R.l = __shfl_up_sync(0xffffffffu, v[3], 1);    // lane 0: own value (edge column, never an output)
  R.r = __shfl_down_sync(0xffffffffu, v[0], 1);  // lane 31: own value (edge column, never an output)
  return R;
}

// neighbourhood of column k from rows S (y-1), M (y), N (y+1)
__device__ __forceinline__ Nb<float> nb6(const Row6& S, const Row6& M, const Row6& N, int k) {
  Nb<float> nb;
  nb.c = M.v[k];
  nb.we = r6(M, k - 1) + r6(M, k + 1);
  nb.ns = S.v[k] + N.v[k];
  nb.d1 = r6(N, k - 1) + r6(S, k + 1);  // NW + SE
  nb.d2 = r6(N, k + 1) + r6(S, k - 1);  // NE + SW
  return nb;
}

// Load 4 columns x0..x0+3 of row y (zeros outside [0,n)^2 or when base is null).
__device__ __forceinline__ void load4(const float* base, int ld, int y, int x0, int n, float (&out)[4]) {
  if (base == nullptr || (unsigned)y >= (unsigned)n || x0 >= n || x0 + 3 < 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = 0.f;
    return;
  }
  const float* p = base + (size_t)y * ld;
  if (x0 >= 0) {  // x0 is a multiple of 4 and x0 + 3 < pitch: one aligned 16-byte load
    const float4 q = *reinterpret_cast<const float4*>(p + x0);
    out[0] = q.x; out[1] = x0 + 1 < n ? q.y : 0.f; out[2] = x0 + 2 < n ? q.z : 0.f; out[3] = x0 + 3 < n ? q.w : 0.f;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = 0.f;
  }
}

// ---------------------------------------------------------------------------------------------
// Pass B: v <- v + P v_c, nu Jacobi sweeps (nu <= 2), optional residual partial sums.
// ---------------------------------------------------------------------------------------------
// Coarse row J interpolated in x to this lane's 4 fine columns (zeros outside the coarse grid).
__device__ __forceinline__ void coarse_row_x(const float* vc, int ldc, int J, int nc, int x0, float (&out)[4]) {
  // fine x0 (even) lies between coarse x0/2-1 and x0/2; x0+1 on coarse x0/2; x0+2 between x0/2 and
  // x0/2+1; x0+3 on coarse x0/2+1
  const int I = x0 >> 1;
  float p0 = 0.f, p1 = 0.f;
  if ((unsigned)J < (unsigned)nc && x0 >= 0 && I < nc) {
    const float* q = vc + (size_t)J * ldc + I;
    if (I + 1 < nc) {
      const float2 t = *reinterpret_cast<const float2*>(q);
      p0 = t.x; p1 = t.y;
    } else {
      p0 = q[0];
    }
  }
  const float pl = __shfl_up_sync(0xffffffffu, p1, 1);  // coarse x0/2 - 1 (from the lane to the left)
  const float left = (x0 >= 2) ? pl : 0.f;
  out[0] = 0.5f * (left + p0);
  out[1] = p0;
  out[2] = 0.5f * (p0 + p1);
  out[3] = p1;
}

template <int NU, bool NORM>
__global__ void __launch_bounds__(32 * SF_WARPS) pass_b_stream_f32(const PassBArgs<float> a, int R) {
  if (a.skip && *a.skip) return;
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * SF_WARPS + (threadIdx.x >> 5);
  const int n = a.n, nc = (n - 1) / 2;
  const int xs = strip * SF_COLS;
  const int ys = blockIdx.y * R;
  const int x0 = xs - 4 + 4 * lane;
  double ss = 0.0;
  if (xs < n) {
    const Coef<float> c = load_coef(a.coef, a.level);
    const bool out_lane = lane >= 1 && lane <= 30;
    bool colin[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) colin[k] = (unsigned)(x0 + k) < (unsigned)n;
    constexpr int DEPTH = NU + (NORM ? 1 : 0);
    Row6 w[DEPTH + 1][3];
    float fdel[DEPTH + 1][4];
#pragma unroll
    for (int s = 0; s <= DEPTH; ++s)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        w[s][r].l = w[s][r].r = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) w[s][r].v[k] = 0.f;
      }
#pragma unroll
    for (int d = 0; d <= DEPTH; ++d)
#pragma unroll
      for (int k = 0; k < 4; ++k) fdel[d][k] = 0.f;
    const int y_first = ys - DEPTH - 1;
    const int steps = R + 2 * DEPTH + 2;
    // interpolated coarse rows: cr_lo = coarse row J_lo, cr_hi = J_lo + 1 (x-interpolated)
    float qv[SF_AHEAD_B][4], qf[SF_AHEAD_B][4];
#pragma unroll
    for (int r = 0; r < SF_AHEAD_B; ++r) {
      load4(a.vin, a.ldvin, y_first + r, x0, n, qv[r]);
      load4(a.f, a.ldf, y_first + r, x0, n, qf[r]);
    }
    // unrolled by the period of the register windows (3) so their shifts become register renames
#pragma unroll 3
  for (int t = 0; t < steps; ++t) {
      const int y_in = y_first + t;
      float cv[4], cf[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) { cv[k] = qv[0][k]; cf[k] = qf[0][k]; }
#pragma unroll
      for (int r = 0; r + 1 < SF_AHEAD_B; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) { qv[r][k] = qv[r + 1][k]; qf[r][k] = qf[r + 1][k]; }
      if (t + SF_AHEAD_B < steps) {
        load4(a.vin, a.ldvin, y_in + SF_AHEAD_B, x0, n, qv[SF_AHEAD_B - 1]);
        load4(a.f, a.ldf, y_in + SF_AHEAD_B, x0, n, qf[SF_AHEAD_B - 1]);
      }
      // stage 0: corrected row y_in = v + P v_c (fine odd rows sit on coarse row (y-1)/2; even rows
      // average coarse rows y/2 - 1 and y/2)
      float corr[4];
      if ((unsigned)y_in < (unsigned)n) {
        float ca[4];
        if (y_in & 1) {
          coarse_row_x(a.vc, a.ldc, y_in >> 1, nc, x0, ca);
#pragma unroll
          for (int k = 0; k < 4; ++k) corr[k] = colin[k] ? cv[k] + ca[k] : 0.f;
        } else {
          float cb[4];
          coarse_row_x(a.vc, a.ldc, (y_in >> 1) - 1, nc, x0, ca);
          coarse_row_x(a.vc, a.ldc, y_in >> 1, nc, x0, cb);
#pragma unroll
          for (int k = 0; k < 4; ++k) corr[k] = colin[k] ? cv[k] + 0.5f * (ca[k] + cb[k]) : 0.f;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) corr[k] = 0.f;
      }
      w[0][0] = w[0][1];
      w[0][1] = w[0][2];
      w[0][2] = with_halo(corr);
#pragma unroll
      for (int d = DEPTH; d > 0; --d)
#pragma unroll
        for (int k = 0; k < 4; ++k) fdel[d][k] = fdel[d - 1][k];
#pragma unroll
      for (int k = 0; k < 4; ++k) fdel[0][k] = cf[k];
#pragma unroll
      for (int s = 1; s <= DEPTH; ++s) {
        const int ys_out = y_in - s;
        const bool row_in = (unsigned)ys_out < (unsigned)n;
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const Nb<float> nb = nb6(w[s - 1][0], w[s - 1][1], w[s - 1][2], k);
          const float v = s <= NU ? jacobi_update(nb, fdel[s][k], c) : residual_at(nb, fdel[s][k], c);
          o[k] = (row_in && colin[k]) ? v : 0.f;
        }
        w[s][0] = w[s][1];
        w[s][1] = w[s][2];
        w[s][2] = with_halo(o);
      }
      const int yv = y_in - NU;  // relaxed output row
      if (out_lane && yv >= ys && yv < ys + R && yv < n && x0 < n) {
        const Row6& o = w[NU][2];
        float* p = a.vout + (size_t)yv * a.ldvout + x0;
        if (x0 + 3 < n) {
          *reinterpret_cast<float4*>(p) = make_float4(o.v[0], o.v[1], o.v[2], o.v[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (colin[k]) p[k] = o.v[k];
        }
      }
      if (NORM) {
        const int yr = y_in - DEPTH;
        if (out_lane && yr >= ys && yr < ys + R && yr < n) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (colin[k]) {
              const double r = (double)w[DEPTH][2].v[k];
              ss = fma(r, r, ss);
            }
        }
      }
    }
  }
  if (NORM) {
    __shared__ double red[SF_WARPS];
    const double t = block_sum<32 * SF_WARPS>(ss, red);
    if (threadIdx.x == 0) a.partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

}  // namespace kc

namespace kc {

// ---------------------------------------------------------------------------------------------
// FP32 tile passes staged in shared memory (the large FP32 levels). A CTA owns a TX x TY tile of
// outputs (TX = 112, TY = 16) and stages the tile with a halo of 8 columns and 4 rows on each side:
// 128 x 24 floats per field, loaded with float4 (zeros outside the grid). A stage (a sweep, the
// residual) is computed row by row, one warp per row: lane q owns the four columns 4q..4q+3, keeps
// the rows above and below in registers as the warp walks down its band of rows, and gets its
// left and right neighbours from the adjacent lanes. Points near the staged border are computed
// from incomplete neighbourhoods, but the halo is wider than the region any output depends on.
// Points outside the grid are reset to zero only in tiles that touch its edge. About half the
// instructions per point of the register pipelines (which keep every stage's rows in registers).
// ---------------------------------------------------------------------------------------------
constexpr int T32_TX = 112, T32_TY = 16;       // outputs per tile (16 rows: five CTAs per SM)
constexpr int T32_P = 128, T32_R = T32_TY + 8;  // staged row pitch (floats) and rows
constexpr int T32_HX = 8, T32_HY = 4;           // staged halo: columns, rows
constexpr int T32_NT = 256;                     // 8 warps
constexpr size_t T32_FIELD = size_t(T32_P) * T32_R;

__host__ __device__ constexpr size_t tile32_smem_a() { return 3 * T32_FIELD * sizeof(float); }
// pass B: v (two buffers), f, and the coarse rows and columns the tile interpolates from
constexpr int T32_CP = T32_P / 2 + 4, T32_CR = T32_R / 2 + 4;
__host__ __device__ constexpr size_t tile32_smem_b() {
  return (3 * T32_FIELD + size_t(T32_CP) * T32_CR) * sizeof(float);
}

// Stage `src` rows [r0, r1) into `dst` rows [r0, r1): out = Jacobi (RES = false) or residual
// (RES = true) of src with right-hand side f. Warp w takes a contiguous band of rows.
template <bool RES>
__device__ __forceinline__ void tile32_stage(const float* __restrict__ src, const float* __restrict__ f,
                                             float* __restrict__ dst, int r0, int r1, const Coef<float>& c,
                                             bool edge, int gx0, int gy0, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rows = r1 - r0, per = (rows + T32_NT / 32 - 1) / (T32_NT / 32);
  const int a = r0 + warp * per, b = min(r1, a + per);
  if (a >= b) return;
  auto row = [&](int r) {  // 4 columns of staged row r plus the neighbouring column on each side
    Row6 R;
    const float4 q = *reinterpret_cast<const float4*>(src + r * T32_P + 4 * lane);
    R.v[0] = q.x; R.v[1] = q.y; R.v[2] = q.z; R.v[3] = q.w;
    R.l = __shfl_up_sync(0xffffffffu, q.w, 1);    // lane 0: its own value (a border column)
    R.r = __shfl_down_sync(0xffffffffu, q.x, 1);  // lane 31: its own value (a border column)
    return R;
  };
  Row6 S = row(a - 1), M = row(a);
  for (int r = a; r < b; ++r) {
    const Row6 N = row(r + 1);
    const float4 fq = *reinterpret_cast<const float4*>(f + r * T32_P + 4 * lane);
    const float fv[4] = {fq.x, fq.y, fq.z, fq.w};
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const Nb<float> nb = nb6(S, M, N, k);
      o[k] = RES ? residual_at(nb, fv[k], c) : jacobi_update(nb, fv[k], c);
    }
    if (edge) {  // outside the grid the field stays zero
      const int gy = gy0 + r;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int gx = gx0 + 4 * lane + k;
        if ((unsigned)gy >= (unsigned)n || (unsigned)gx >= (unsigned)n) o[k] = 0.f;
      }
    }
    *reinterpret_cast<float4*>(dst + r * T32_P + 4 * lane) = make_float4(o[0], o[1], o[2], o[3]);
    S = M;
    M = N;
  }
}

// Stage rows of `base` (ld floats per row; nullptr: zeros) into a T32_R x T32_P field.
__device__ __forceinline__ void tile32_load(const float* base, int ld, float* dst, int gx0, int gy0, int n) {
  for (int e = threadIdx.x; e < T32_R * (T32_P / 4); e += T32_NT) {
    const int r = e / (T32_P / 4), q = e - r * (T32_P / 4);
    const int gy = gy0 + r, gx = gx0 + 4 * q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (base && (unsigned)gy < (unsigned)n && gx >= 0 && gx < n) {
      const float* p = base + (size_t)gy * ld + gx;
      if (gx + 3 < n) {
        v = *reinterpret_cast<const float4*>(p);
      } else {
        v.x = p[0];
        if (gx + 1 < n) v.y = p[1];
        if (gx + 2 < n) v.z = p[2];
      }
    }
    *reinterpret_cast<float4*>(dst + r * T32_P + 4 * q) = v;
  }
}

// Pass A (nu <= 2 sweeps, residual, full weighting) on one tile; the same PassAArgs as the other
// pass A kernels. Arrays 16-byte aligned with pitches that are multiples of 4 floats.
template <int NU>
__global__ void __launch_bounds__(T32_NT) pass_a_tile32(const PassAArgs<float> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* fs = reinterpret_cast<float*>(smem_raw);
  float* b0 = fs + T32_FIELD;
  float* b1 = b0 + T32_FIELD;
  const int n = a.n, nc = (n - 1) / 2;
  const int x0 = blockIdx.x * T32_TX, y0 = blockIdx.y * T32_TY;
  const int gx0 = x0 - T32_HX, gy0 = y0 - T32_HY;
  const bool edge = gx0 < 0 || gy0 < 0 || gx0 + T32_P > n || gy0 + T32_R > n;
  const Coef<float> c = load_coef(a.coef, a.level);
  tile32_load(a.f, a.ldf, fs, gx0, gy0, n);
  if (a.vin || NU == 0) tile32_load(a.vin, a.ldvin, b0, gx0, gy0, n);  // nullptr: zeros
  __syncthreads();
  float* src = b0;
  float* dst = b1;
#pragma unroll
  for (int s = 1; s <= NU; ++s) {
    if (s == 1 && a.vin == nullptr) {
      // from a zero start the first sweep is v = w f (the update of v = 0)
      for (int e = threadIdx.x; e < (T32_R - 2) * (T32_P / 4); e += T32_NT) {
        const int r = 1 + e / (T32_P / 4), q = e - (r - 1) * (T32_P / 4);
        const float4 fq = *reinterpret_cast<const float4*>(fs + r * T32_P + 4 * q);
        // fs is zero outside the grid, so w f is too
        *reinterpret_cast<float4*>(dst + r * T32_P + 4 * q) = make_float4(c.w * fq.x, c.w * fq.y, c.w * fq.z, c.w * fq.w);
      }
    } else {
      tile32_stage<false>(src, fs, dst, s, T32_R - s, c, edge, gx0, gy0, n);
    }
    __syncthreads();
    float* t = src; src = dst; dst = t;
  }
  // relaxed v: rows [HY, HY + TY), columns [HX, HX + TX) of src
  if (a.vout) {
    for (int e = threadIdx.x; e < T32_TY * (T32_TX / 4); e += T32_NT) {
      const int r = e / (T32_TX / 4), q = e - r * (T32_TX / 4);
      const int gy = y0 + r, gx = x0 + 4 * q;
      if (gy < n && gx < n) {
        const float4 v = *reinterpret_cast<const float4*>(src + (T32_HY + r) * T32_P + T32_HX + 4 * q);
        float* p = a.vout + (size_t)gy * a.ldvout + gx;
        if (gx + 3 < n) {
          *reinterpret_cast<float4*>(p) = v;
        } else {
          p[0] = v.x;
          if (gx + 1 < n) p[1] = v.y;
          if (gx + 2 < n) p[2] = v.z;
        }
      }
    }
  }
  // residual on rows [HY - 1, HY + TY + 1) (full weighting reads one row above and below)
  tile32_stage<true>(src, fs, dst, T32_HY - 1, T32_HY + T32_TY + 1, c, edge, gx0, gy0, n);
  __syncthreads();
  // coarse point (I, J) on fine (2I+1, 2J+1); this tile owns I in [x0/2, x0/2 + TX/2), J likewise
  for (int e = threadIdx.x; e < (T32_TY / 2) * (T32_TX / 2); e += T32_NT) {
    const int j = e / (T32_TX / 2), i = e - j * (T32_TX / 2);
    const int I = x0 / 2 + i, J = y0 / 2 + j;
    if (I < nc && J < nc) {
      const int k = (T32_HY + 2 * j + 1) * T32_P + (T32_HX + 2 * i + 1);
      a.fc[(size_t)J * a.ldc + I] = full_weight(dst, k, T32_P);
    }
  }
}

// Pass B (v + P v_c, nu <= 2 sweeps; no residual sums) on one tile.
template <int NU>
__global__ void __launch_bounds__(T32_NT) pass_b_tile32(const PassBArgs<float> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* fs = reinterpret_cast<float*>(smem_raw);
  float* b0 = fs + T32_FIELD;
  float* b1 = b0 + T32_FIELD;
  float* cs = b1 + T32_FIELD;  // coarse region: rows cy0.., columns cx0.., pitch T32_CP
  const int n = a.n, nc = (n - 1) / 2;
  const int x0 = blockIdx.x * T32_TX, y0 = blockIdx.y * T32_TY;
  const int gx0 = x0 - T32_HX, gy0 = y0 - T32_HY;
  const bool edge = gx0 < 0 || gy0 < 0 || gx0 + T32_P > n || gy0 + T32_R > n;
  const Coef<float> c = load_coef(a.coef, a.level);
  // coarse points that interpolation to fine [gx0, gx0 + P) x [gy0, gy0 + R) reads
  const int cx0 = (gx0 >> 1) - 1, cy0 = (gy0 >> 1) - 1;
  for (int e = threadIdx.x; e < T32_CR * T32_CP; e += T32_NT) {
    const int r = e / T32_CP, q = e - r * T32_CP;
    const int cy = cy0 + r, cx = cx0 + q;
    cs[e] = ((unsigned)cy < (unsigned)nc && (unsigned)cx < (unsigned)nc) ? a.vc[(size_t)cy * a.ldc + cx] : 0.f;
  }
  tile32_load(a.f, a.ldf, fs, gx0, gy0, n);
  tile32_load(a.vin, a.ldvin, b0, gx0, gy0, n);
  __syncthreads();
  // corrected v = v + P v_c on every staged point inside the grid, four columns at a time: fine
  // columns gx..gx+3 (gx even) lie between coarse gx/2 - 1 and gx/2, on gx/2, between gx/2 and
  // gx/2 + 1, on gx/2 + 1; odd rows on coarse row (gy - 1)/2, even rows between gy/2 - 1 and gy/2
  for (int e = threadIdx.x; e < T32_R * (T32_P / 4); e += T32_NT) {
    const int r = e / (T32_P / 4), q = e - r * (T32_P / 4);
    const int gy = gy0 + r, gx = gx0 + 4 * q;
    if ((unsigned)gy >= (unsigned)n) continue;
    const int hx = (gx >> 1) - cx0, hy = (gy >> 1) - cy0;
    auto xrow = [&](int row, float (&o)[4]) {
      const float* cr = cs + row * T32_CP + hx;
      const float l = cr[-1], p0 = cr[0], p1 = cr[1];
      o[0] = 0.5f * (l + p0);
      o[1] = p0;
      o[2] = 0.5f * (p0 + p1);
      o[3] = p1;
    };
    float corr[4];
    if (gy & 1) {
      xrow(hy, corr);
    } else {
      float ca[4], cb[4];
      xrow(hy - 1, ca);
      xrow(hy, cb);
#pragma unroll
      for (int k = 0; k < 4; ++k) corr[k] = 0.5f * (ca[k] + cb[k]);
    }
    if (edge) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if ((unsigned)(gx + k) >= (unsigned)n) corr[k] = 0.f;
    }
    float4* pv = reinterpret_cast<float4*>(b0 + r * T32_P + 4 * q);
    float4 v = *pv;
    v.x += corr[0]; v.y += corr[1]; v.z += corr[2]; v.w += corr[3];
    *pv = v;
  }
  __syncthreads();
  float* src = b0;
  float* dst = b1;
#pragma unroll
  for (int s = 1; s <= NU; ++s) {
    tile32_stage<false>(src, fs, dst, s, T32_R - s, c, edge, gx0, gy0, n);
    __syncthreads();
    float* t = src; src = dst; dst = t;
  }
  for (int e = threadIdx.x; e < T32_TY * (T32_TX / 4); e += T32_NT) {
    const int r = e / (T32_TX / 4), q = e - r * (T32_TX / 4);
    const int gy = y0 + r, gx = x0 + 4 * q;
    if (gy < n && gx < n) {
      const float4 v = *reinterpret_cast<const float4*>(src + (T32_HY + r) * T32_P + T32_HX + 4 * q);
      float* p = a.vout + (size_t)gy * a.ldvout + gx;
      if (gx + 3 < n) {
        *reinterpret_cast<float4*>(p) = v;
      } else {
        p[0] = v.x;
        if (gx + 1 < n) p[1] = v.y;
        if (gx + 2 < n) p[2] = v.z;
      }
    }
  }
}

}  // namespace kc
