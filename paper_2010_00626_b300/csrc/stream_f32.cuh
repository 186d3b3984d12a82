// FP32 fused level passes written as register pipelines (the FP32 cycle of the mixed forms).
//
// FP32 level passes are bound by HBM bandwidth and instruction issue, not by arithmetic: the
// shared-memory tile kernels spend their issue slots on index arithmetic and barriers. Here one
// warp owns a vertical strip of 128 columns (4 consecutive columns per lane, read with float4 loads)
// and streams down a chunk of rows. Every stage of the pass (Jacobi sweeps, residual, full
// weighting; or interpolation + sweeps) keeps a window of three rows in registers and gets the
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
constexpr int SF_AHEAD = 3;   // input rows loaded ahead of use (pass A)
constexpr int SF_AHEAD_B = 4; // same for pass B (at 4095^2: 115 -> 107 us; pass A got slower at 4)

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
// Pass A: nu Jacobi sweeps (nu <= 2), residual, full weighting. One warp: output columns
// [xs, xs+120) of rows [ys, ys+R).
// ---------------------------------------------------------------------------------------------
template <int NU>
__global__ void __launch_bounds__(32 * SF_WARPS) pass_a_stream_f32(const PassAArgs<float> a, int R) {
  if (a.skip && *a.skip) return;
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * SF_WARPS + (threadIdx.x >> 5);
  const int n = a.n, nc = (n - 1) / 2;
  const int xs = strip * SF_COLS;
  if (xs >= n) return;  // uniform per warp
  const int ys = blockIdx.y * R;
  const int x0 = xs - 4 + 4 * lane;
  const Coef<float> c = load_coef(a.coef, a.level);
  const bool out_lane = lane >= 1 && lane <= 30;  // owns output columns x0..x0+3
  bool colin[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) colin[k] = (unsigned)(x0 + k) < (unsigned)n;

  // stage windows (south, middle, north) and delayed right-hand sides
  constexpr int DEPTH = NU + 1;            // stages before the restriction: NU sweeps + residual
  Row6 w[DEPTH + 1][3];                    // w[0]: input rows; w[s]: output rows of stage s
  float fdel[DEPTH + 1][4];                // fdel[d]: f of input row y_in - d
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

  // residual rows kept for the restriction (vertical weights need rows yr-2, yr-1, yr)
  float rres[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  const int y_first = ys - DEPTH - 1;  // first input row
  const int steps = R + 2 * DEPTH + 2;
  // input rows are loaded SF_AHEAD rows ahead of use (bytes in flight hide HBM latency)
  float qv[SF_AHEAD][4], qf[SF_AHEAD][4];
#pragma unroll
  for (int r = 0; r < SF_AHEAD; ++r) {
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
    for (int r = 0; r + 1 < SF_AHEAD; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k) { qv[r][k] = qv[r + 1][k]; qf[r][k] = qf[r + 1][k]; }
    if (t + SF_AHEAD < steps) {
      load4(a.vin, a.ldvin, y_in + SF_AHEAD, x0, n, qv[SF_AHEAD - 1]);
      load4(a.f, a.ldf, y_in + SF_AHEAD, x0, n, qf[SF_AHEAD - 1]);
    }
    // input window and f delay line
    w[0][0] = w[0][1];
    w[0][1] = w[0][2];
    w[0][2] = with_halo(cv);
#pragma unroll
    for (int d = DEPTH; d > 0; --d)
#pragma unroll
      for (int k = 0; k < 4; ++k) fdel[d][k] = fdel[d - 1][k];
#pragma unroll
    for (int k = 0; k < 4; ++k) fdel[0][k] = cf[k];
    // stages: stage s produces row y_in - s from the window of stage s-1 (rows y_in-s-1 .. y_in-s+1)
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
    // relaxed v: output row y_in - NU (the last sweep)
    {
      const int yv = y_in - NU;
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
    }
    // restriction: the residual row just produced is yr = y_in - DEPTH; coarse row J sits on fine
    // row 2J+1 = yr - 1 and weighs residual rows yr-2, yr-1, yr by 1, 2, 1
    {
      const int yr = y_in - DEPTH;
      const Row6& rn = w[DEPTH][2];
      const int yc = yr - 1;
      if ((yc & 1) && yc >= ys && yc < ys + R && yc < n) {
        float vs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) vs[k] = rres[0][k] + 2.f * rres[1][k] + rn.v[k];
        const float right = __shfl_down_sync(0xffffffffu, vs[0], 1);
        // this lane's odd columns x0+1 and x0+3 are coarse points (x0 is a multiple of 4)
        const float c1 = 0.0625f * (vs[0] + 2.f * vs[1] + vs[2]);
        const float c3 = 0.0625f * (vs[2] + 2.f * vs[3] + right);
        const int J = (yc - 1) >> 1, I = x0 >> 1;
        if (out_lane && J < nc && I < nc) {
          float* q = a.fc + (size_t)J * a.ldc + I;
          if (I + 1 < nc) *reinterpret_cast<float2*>(q) = make_float2(c1, c3);
          else q[0] = c1;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        rres[0][k] = rres[1][k];
        rres[1][k] = rn.v[k];
      }
    }
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
