// Many right-hand sides at once (backward-Euler time steps of an RC grid).
//
// The same VTM sweep (Sec. VI, Eq. 11/14) for R right-hand sides: per
// sub-circuit the wave update is a dense product W_out = T_P W_in + C_P with
// W_in = the R incident waves of every port (p x R).  Vectors are kept
// row-major, [port][R] and [node][R], so that the exchange moves one
// contiguous row per port.
//
// Kernels:
//  * batch_band_solve_kernel: K_P^-1 V for a block of RG right-hand sides,
//    one thread per band offset (each thread updates its row for RG
//    columns), factor columns prefetched D steps ahead;
//  * batch_sweep_kernel: one CTA per (tile, block of 64 outputs); each
//    thread owns a 4 x 4 block of (output, RHS); T and the gathered incident
//    waves pass through shared memory in chunks of 16 inputs; the residual of
//    the previous sweep (per RHS) is reduced per item and then over items in
//    a fixed order;
//  * batch_sweep_mma_kernel: the same with BF16 T and BF16 incident waves on
//    the tensor cores (mma.sync m16n8k16, FP32 accumulate).
#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "ptx.h"
#include "vtm_internal.h"

namespace vtm {

struct BatchCtrl {
  int k;
  int flag;  // 0 running, 1 converged, 2 sweep limit, 3 diverged, 4 stalled
  unsigned counter;
  unsigned work;   // next entry of the work list (persistent CTAs)
  int conv_sweep;
  int k_max;
  int best_k;
  int stall;
  int R;
  double best_ratio;  // max over columns of res2 / tol2 at best_k
  double first_ratio;
};

// sum of p[0], p[stride], ... p[(n-1) stride] (rows written by other CTAs of
// this launch: read through L2) with four interleaved accumulators, so that
// four loads are in flight per step; the order depends on n only
__device__ __forceinline__ double ordered_sum_strided(const double* p, int n, int stride) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
    a0 += __ldcg(p + (size_t)k * stride);
    a1 += __ldcg(p + (size_t)(k + 1) * stride);
    a2 += __ldcg(p + (size_t)(k + 2) * stride);
    a3 += __ldcg(p + (size_t)(k + 3) * stride);
  }
  for (; k < n; ++k) a0 += __ldcg(p + (size_t)k * stride);
  return (a0 + a1) + (a2 + a3);
}

// ---------------------------------------------------------------------------
// permutation between the caller's column-major n x R and [pos][R]
// ---------------------------------------------------------------------------

// Permuted FP64 vectors are column-major too, V[r * n + pos], so both sides
// of the permutation are read and written along a column (the FP32 vectors of
// the low-precision path are row-major: see batch_gather_rm_kernel).
template <class FT>
__global__ void batch_gather_kernel(const int32_t* __restrict__ perm, const double* __restrict__ src,
                                    FT* __restrict__ dst, int64_t n, int R) {
  const int64_t total = n * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n, pos = i % n;
    dst[i] = (FT)src[r * n + perm[pos]];
  }
}

// dst[r][node] (+)= src[r][iperm[node]]: written along the caller's order,
// read through the inverse permutation (one column at a time stays in L2)
template <class FT>
__global__ void batch_scatter_kernel(const int32_t* __restrict__ iperm, const FT* __restrict__ src,
                                     double* __restrict__ dst, int64_t n, int R, int accumulate) {
  const int64_t total = n * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n, node = i % n;
    const double v = (double)src[r * n + iperm[node]];
    if (accumulate) dst[i] += v;
    else dst[i] = v;
  }
}

// r = b - A x for R columns at once (column-major), with ||r_c||^2 and
// ||b_c||^2 per column.  Block b covers column group by = b % gy (columns
// 8 by .. 8 by + 7) and rows bx, bx + gx, ... (units of 256 rows), bx = b /
// gy: the groups of one row range run side by side, so each row of A comes
// from DRAM once.  Per row, the products of one nonzero with the 8 columns
// are independent loads.  Per-block partial sums, then the last block of
// each group adds them in a fixed order.  counters[by] start at 0 and are
// left at 0; out[2 c] = ||r_c||^2, out[2 c + 1] = ||b_c||^2.
__global__ void __launch_bounds__(256) batch_residual_norms_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ x, const double* __restrict__ b,
    double* __restrict__ r, int64_t n, int R, int gx, int gy, double* __restrict__ partials,
    unsigned* __restrict__ counters, double* __restrict__ out) {
  constexpr int CG = 8;
  __shared__ double red[2 * CG][8];
  __shared__ bool last;
  const int by = blockIdx.x % gy, bx = blockIdx.x / gy;
  const int c0 = by * CG;
  const int nc = min(CG, R - c0);
  const double* xg = x + (int64_t)c0 * n;
  const double* bg = b + (int64_t)c0 * n;
  double rr[CG], bb[CG];
#pragma unroll
  for (int c = 0; c < CG; ++c) rr[c] = bb[c] = 0.0;
  for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gx * blockDim.x) {
    const int64_t q0 = rowptr[i], q1 = rowptr[i + 1];
    double acc[CG], bi[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) acc[c] = bi[c] = c < nc ? bg[(int64_t)c * n + i] : 0.0;
    for (int64_t q = q0; q < q1; ++q) {
      const int64_t j = col[q];
      const double v = val[q];
#pragma unroll
      for (int c = 0; c < CG; ++c)
        if (c < nc) acc[c] -= v * xg[(int64_t)c * n + j];
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      if (c < nc) {
        if (r) r[(int64_t)(c0 + c) * n + i] = acc[c];
        rr[c] += acc[c] * acc[c];
        bb[c] += bi[c] * bi[c];
      }
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < CG; ++c) {
    double a = rr[c], e = bb[c];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      e += __shfl_down_sync(0xffffffffu, e, o);
    }
    if (l == 0) {
      red[c][w] = a;
      red[CG + c][w] = e;
    }
  }
  __syncthreads();
  const size_t pb = ((size_t)by * gx + bx) * 2 * CG;
  if (threadIdx.x < 2 * CG) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
    partials[pb + threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&counters[by], 1u) == (unsigned)gx - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 2 * CG) {
    const double t = ordered_sum_strided(partials + (size_t)by * gx * 2 * CG + threadIdx.x, gx, 2 * CG);
    const int c = threadIdx.x % CG;
    if (c < nc) out[2 * (c0 + c) + (threadIdx.x >= CG ? 1 : 0)] = t;
  }
  if (threadIdx.x == 0) counters[by] = 0u;
}

// ---------------------------------------------------------------------------
// double-float residuals of the low-precision batched solves
// ---------------------------------------------------------------------------
//
// GB300's FP64 pipe is narrow: b - A x in FP64 for 64 columns costs about
// seven FP64 FMAs per nonzero and column.  The low-precision refinement
// only needs the residual to about 1e-14 of ||b|| (it is rounded to FP32 as
// the next right-hand side, and its norm decides convergence at 1e-10), so
// it runs in double-float arithmetic on the FP32 pipes instead: A's values
// split once into (h, l) pairs, each column of b and of the iterate scaled by
// 2^-f_c (f_c = the exponent of max |b_c|, an exact scale that keeps every
// double-float within FP32's exponent range) and split by their bits.

// emax[c] = max over the column of the biased exponent of b (emax zeroed)
__global__ void batch_colexp_kernel(const double* __restrict__ b, int64_t n, int R, int* __restrict__ emax) {
  const int c = blockIdx.y;
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)((__double_as_longlong(b[(int64_t)c * n + i]) >> 52) & 0x7ff));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&emax[c], m);
}

// dst[pos][r] = src[r][pos] 2^-f[r] as double-floats: the caller's
// column-major b into the row-major [n][R] layout of the double-float
// vectors, through a shared-memory tile of 32 rows x R
__global__ void __launch_bounds__(256) batch_split_rm_kernel(const double* __restrict__ src,
                                                             const int* __restrict__ f,
                                                             float2* __restrict__ dst, int64_t n, int R) {
  __shared__ float2 tile[32][65];
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int nn = (int)(n - n0 < 32 ? n - n0 : 32);
  const int nl = threadIdx.x & 31;
  if (nl < nn)
    for (int r = threadIdx.x >> 5; r < R; r += 8) tile[nl][r] = df_from_double(src[(int64_t)r * n + n0 + nl], f[r]);
  __syncthreads();
  for (int e = threadIdx.x; e < nn * R; e += blockDim.x) dst[n0 * R + e] = tile[e / R][e % R];
}

// dst = src as double-floats (A's values, no scale)
__global__ void batch_split_kernel(const double* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = df_from_double(src[i], 0);
}

// r' = b' - A x' for up to 64 scaled columns (b', x', r' row-major, [n][R];
// x' = nullptr: x = 0), with ||r'_c||^2 and ||b'_c||^2, in double-float
// arithmetic (Dot2 accumulation seeded with b', paired FP32 instructions for
// two columns at a time).  The lanes lie along the rows: with CG columns per
// lane, LPR = 64 / CG lanes share a row (row slot l / LPR, columns CG (l %
// LPR) .. + CG - 1), so one load instruction of the warp reads 32 / LPR whole
// 512-byte rows of x' (64 columns) and a row's nonzeros serve its LPR lanes.
// One group of up to 64 columns; block bx covers 8 (32 / LPR) rows per step.
// CG = 4 (64 registers, four CTAs per SM) measured faster than CG = 8 (128
// registers, two).  Squares: FP32 per thread and across the lanes of a column, FP64 from
// the warp sums on, blocks added in a fixed order by the last block.
// out[2 c] = ||r'_c||^2, out[2 c + 1] = ||b'_c||^2; counter 0 on entry, left 0.
// r', rounded to FP32 (h + l), goes to the rows iperm[i] of v1 and v2 (when
// given): the right-hand sides of the step's two band solves in the band
// order.
template <int CG, int MINB>
__global__ void __launch_bounds__(256, MINB) batch_residual_rows_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const float2* __restrict__ vdf, const float2* __restrict__ xdf, const float2* __restrict__ bdf,
    const int32_t* __restrict__ iperm, float* __restrict__ v1,
    float* __restrict__ v2, int64_t n, int R, int gx, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ out) {
  constexpr int NP = CG / 2, LPR = 64 / CG, RPW = 32 / LPR;  // lanes per row, rows per warp
  static_assert(CG % 4 == 0, "column group of whole 16-byte FP32 groups");
  __shared__ float red[128][8];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = CG * (lane % LPR);
  const int nc = max(0, min(CG, R - c0));
  const bool vec = nc == CG && (R & 1) == 0;
  const bool vec4 = nc == CG && (R & 3) == 0;  // 16-byte FP32 row stores
  // STREAM: b', read once, marked evict-first, so that the rows of x' the
  // neighbouring rows reuse stay in L2
  auto ld_row = [&](const float2* p, float2 (&o)[CG], bool stream) {
    if (vec) {
#pragma unroll
      for (int c = 0; c < CG; c += 2) {
        const float4 q = stream ? __ldcs(reinterpret_cast<const float4*>(p + c))
                                : *reinterpret_cast<const float4*>(p + c);
        o[c] = make_float2(q.x, q.y);
        o[c + 1] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int c = 0; c < CG; ++c) o[c] = c < nc ? p[c] : make_float2(0.f, 0.f);
    }
  };
  float rr[CG], bb[CG];
#pragma unroll
  for (int c = 0; c < CG; ++c) rr[c] = bb[c] = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * (8 * RPW) + warp * RPW + lane / LPR; i < n;
       i += (int64_t)gx * (8 * RPW)) {
    dacc2 acc[NP];
    const int pos = v1 ? iperm[i] : 0;
    {
      float2 bv[CG];
      ld_row(bdf + i * R + c0, bv, true);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        acc[p].S = make_float2(bv[2 * p].x, bv[2 * p + 1].x);
        acc[p].E = make_float2(bv[2 * p].y, bv[2 * p + 1].y);
        bb[2 * p] += bv[2 * p].x * bv[2 * p].x;
        bb[2 * p + 1] += bv[2 * p + 1].x * bv[2 * p + 1].x;
      }
    }
    if (xdf && nc > 0) {
      // the iterate's row one nonzero ahead, the column index two ahead
      const int64_t q0 = rowptr[i], q1 = rowptr[i + 1];
      float2 xv[CG], a = make_float2(0.f, 0.f), an = make_float2(0.f, 0.f);
      int64_t jn = 0;
      if (q0 < q1) {
        a = vdf[q0];
        ld_row(xdf + (int64_t)col[q0] * R + c0, xv, false);
      }
      if (q0 + 1 < q1) {
        jn = col[q0 + 1];
        an = vdf[q0 + 1];
      }
      for (int64_t q = q0; q < q1; ++q) {
        float2 xn[CG];
        const bool more = q + 1 < q1;
        if (more) ld_row(xdf + jn * R + c0, xn, false);
        int64_t jnn = 0;
        float2 ann = make_float2(0.f, 0.f);
        if (q + 2 < q1) {
          jnn = col[q + 2];
          ann = vdf[q + 2];
        }
        const float2 ah = make_float2(-a.x, -a.x), al = make_float2(-a.y, -a.y);
#pragma unroll
        for (int p = 0; p < NP; ++p)
          dacc2_fma(acc[p], ah, al, make_float2(xv[2 * p].x, xv[2 * p + 1].x),
                    make_float2(-xv[2 * p].x, -xv[2 * p + 1].x), make_float2(xv[2 * p].y, xv[2 * p + 1].y));
        if (more) {
#pragma unroll
          for (int c = 0; c < CG; ++c) xv[c] = xn[c];
          a = an;
        }
        jn = jnn;
        an = ann;
      }
    }
    float2 rv[CG];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const df v = dacc_value(h ? dacc2_hi(acc[p]) : dacc2_lo(acc[p]));
        rv[2 * p + h] = make_float2(v.h, v.l);
        rr[2 * p + h] += v.h * v.h;
      }
    }
    if (v1) {
      float o[CG];
#pragma unroll
      for (int c = 0; c < CG; ++c) o[c] = rv[c].x + rv[c].y;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        float* vp = (k ? v2 : v1);
        if (!vp) continue;
        vp += (int64_t)pos * R + c0;
        if (vec4) {
#pragma unroll
          for (int c = 0; c < CG; c += 4)
            *reinterpret_cast<float4*>(vp + c) = make_float4(o[c], o[c + 1], o[c + 2], o[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < CG; ++c)
            if (c < nc) vp[c] = o[c];
        }
      }
    }
  }
  // per column: the row slots of the warp (lanes l, l + LPR, ...)
#pragma unroll
  for (int c = 0; c < CG; ++c) {
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1) {
      rr[c] += __shfl_xor_sync(0xffffffffu, rr[c], o);
      bb[c] += __shfl_xor_sync(0xffffffffu, bb[c], o);
    }
  }
  if (lane < LPR) {
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      red[c0 + c][warp] = rr[c];
      red[64 + c0 + c][warp] = bb[c];
    }
  }
  __syncthreads();
  if (tid < 128) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += (double)red[tid][k];
    partials[(size_t)blockIdx.x * 128 + tid] = t;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == (unsigned)gx - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid < 128) {
    const double t = ordered_sum_strided(partials + tid, gx, 128);
    const int c = tid & 63;
    if (c < R) out[2 * c + (tid >= 64 ? 1 : 0)] = t;
  }
  if (tid == 0) *counter = 0u;
}

// The FP32 work vectors of the low-precision batched solves are row-major,
// V32[pos][R]: a port's right-hand sides are one contiguous row, so the
// port-wise kernels (injection, port constants) and the band solves' row
// blocks run along rows.  The caller's vectors (and the FP64 path's) stay
// column-major; the two permuting copies transpose through a shared-memory
// tile of 32 positions x R.
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float to_f32(float2 v) { return v.x + v.y; }

// dst[pos][r] = src[r][perm[pos]] rounded to FP32 (src FP64, or a
// double-float pair h + l)
template <class ST>
__global__ void __launch_bounds__(256) batch_gather_rm_kernel(const int32_t* __restrict__ perm,
                                                              const ST* __restrict__ src,
                                                              float* __restrict__ dst, int64_t n, int R) {
  __shared__ float tile[32][65];
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int np = (int)(n - p0 < 32 ? n - p0 : 32);
  const int pl = threadIdx.x & 31;
  if (pl < np) {
    const int64_t node = perm[p0 + pl];
    for (int r = threadIdx.x >> 5; r < R; r += 8) tile[pl][r] = to_f32(src[(int64_t)r * n + node]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < np * R; e += blockDim.x) dst[p0 * R + e] = tile[e / R][e % R];
}

// x[r][node] (+)= d[iperm[node]][r] (DF: times 2^f_r, exact in FP64, and
// x'[node][r] = x 2^-f_r as a double-float, row-major through a second tile)
template <bool DF>
__global__ void __launch_bounds__(256) batch_scatter_rm_kernel(const int32_t* __restrict__ iperm,
                                                               const float* __restrict__ d,
                                                               double* __restrict__ x, float2* __restrict__ xdf,
                                                               const int* __restrict__ f, int64_t n, int R,
                                                               int accumulate) {
  __shared__ float tile[32][65];
  __shared__ float2 tdf[DF ? 32 : 1][DF ? 65 : 1];
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int nn = (int)(n - n0 < 32 ? n - n0 : 32);
  for (int e = threadIdx.x; e < nn * R; e += blockDim.x) {
    const int nl = e / R, r = e % R;
    tile[nl][r] = d[(int64_t)iperm[n0 + nl] * R + r];
  }
  __syncthreads();
  const int nl = threadIdx.x & 31;
  if (nl < nn) {
    for (int r = threadIdx.x >> 5; r < R; r += 8) {
      const int64_t i = (int64_t)r * n + n0 + nl;
      if (DF) {
        const int fr = f[r];
        const double v = double_from_float(tile[nl][r], fr);
        const double xn = accumulate ? x[i] + v : v;
        x[i] = xn;
        tdf[nl][r] = df_from_double(xn, fr);
      } else {
        const double v = (double)tile[nl][r];
        if (accumulate) x[i] += v;
        else x[i] = v;
      }
    }
  }
  if (DF) {
    __syncthreads();
    for (int e = threadIdx.x; e < nn * R; e += blockDim.x) xdf[n0 * R + e] = tdf[e / R][e % R];
  }
}

// V32[pos(node)][r] += sum over the node's ports of beta_s w_in[s][r], in FP32
// (beta in FP32: GB300's FP64 pipe would bound the kernel, and the rounding
// is far below what the FP32 / 16-bit sweeps carry)
__global__ void batch_inject_rm_kernel(const int32_t* __restrict__ port_pos, const uint8_t* __restrict__ run,
                                       const float* __restrict__ beta, const float* __restrict__ st,
                                       float* __restrict__ V, int64_t nports, int R) {
  const int64_t total = nports * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / R;
    const int r = (int)(i % R);
    const int nr = run[s];
    if (!nr) continue;
    float acc = 0.f;
    for (int q = 0; q < nr; ++q) acc = fmaf(beta[s + q], st[(s + q) * 2 * R + r], acc);
    V[(int64_t)port_pos[s] * R + r] += acc;
  }
}

// c[s][r] = (2 W beta_s / d_s) x0[pos(s)][r], x0 row-major FP32, in FP32
__global__ void batch_const_rm_kernel(const int32_t* __restrict__ port_pos, const float* __restrict__ bout,
                                      const float* __restrict__ x0, float* __restrict__ c, int64_t nports,
                                      int R) {
  const int64_t total = nports * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / R;
    const int r = (int)(i % R);
    c[i] = bout[s] * x0[(int64_t)port_pos[s] * R + r];
  }
}

// ---------------------------------------------------------------------------
// band solves for RG right-hand sides per CTA
// ---------------------------------------------------------------------------
//
// V[pos][R] in global memory, the tile's block of RG columns staged in
// shared memory (column-major).  Thread a (1..bw) owns band offset a: at step j
// it updates row j + a with multiplier Lc[j][a] (forward) or row j - a with
// Uc[j][a] (backward); one barrier per step.  Each thread prefetches its
// multiplier D columns ahead.

template <class FT, int RG, int D>
__global__ void batch_band_solve_kernel(const int32_t* __restrict__ node_off,
                                        const int32_t* __restrict__ bwv,
                                        const int64_t* __restrict__ band_off,
                                        const FT* __restrict__ Lc, const FT* __restrict__ Uc,
                                        FT* __restrict__ V, int R, int64_t rs, int64_t cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ngroups = (R + RG - 1) / RG;
  const int t = blockIdx.x / ngroups;
  const int r0 = (blockIdx.x % ngroups) * RG;
  const int rg = min(RG, R - r0);
  const int base = node_off[t];
  const int n = node_off[t + 1] - base;
  const int bw = bwv[t];
  const int B = bw + 1;
  const FT* lc = Lc + band_off[t];
  const FT* uc = Uc + band_off[t];
  const int tid = threadIdx.x;
  // column-major in shared memory, v[c * n + row]: at every step the threads
  // (band offsets) touch consecutive rows of a column, without bank conflicts
  FT* v = reinterpret_cast<FT*>(smem_raw);
  for (int i = tid; i < n * RG; i += blockDim.x) {
    const int c = i / n, row = i % n;
    v[i] = c < rg ? V[(int64_t)(base + row) * rs + (int64_t)(r0 + c) * cs] : FT(0);
  }
  __syncthreads();
  const int a = tid + 1;  // band offset of this thread
  const bool act = a <= bw;
  FT pf[D];
  // forward sweep (scaled multipliers, see band.cuh)
#pragma unroll
  for (int d = 0; d < D; ++d) pf[d] = (act && d < n && a <= n - 1 - d) ? lc[(size_t)d * B + a] : FT(0);
  for (int j0 = 0; j0 < n; j0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = j0 + d;
      if (j < n) {
        if (act && a <= n - 1 - j) {
          const FT m = pf[d];
#pragma unroll
          for (int c = 0; c < RG; ++c) v[c * n + j + a] -= m * v[c * n + j];
        }
        const int jn = j + D;
        pf[d] = (act && jn < n && a <= n - 1 - jn) ? lc[(size_t)jn * B + a] : FT(0);
        __syncthreads();
      }
    }
  }
  for (int i = tid; i < n * RG; i += blockDim.x) v[i] *= lc[(size_t)(i % n) * B];
  __syncthreads();
  // backward sweep
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int j = n - 1 - d;
    pf[d] = (act && j >= 0 && a <= j) ? uc[(size_t)j * B + a] : FT(0);
  }
  for (int j0 = n - 1; j0 >= 0; j0 -= D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = j0 - d;
      if (j >= 0) {
        if (act && a <= j) {
          const FT m = pf[d];
#pragma unroll
          for (int c = 0; c < RG; ++c) v[c * n + j - a] -= m * v[c * n + j];
        }
        const int jn = j - D;
        pf[d] = (act && jn >= 0 && a <= jn) ? uc[(size_t)jn * B + a] : FT(0);
        __syncthreads();
      }
    }
  }
  for (int i = tid; i < n * RG; i += blockDim.x) {
    const int c = i / n, row = i % n;
    if (c < rg) V[(int64_t)(base + row) * rs + (int64_t)(r0 + c) * cs] = v[i] * uc[(size_t)row * B];
  }
}

// The same solve with only a window of WB = bw + 1 + PF rows of the tile's
// column block in shared memory (rows enter PF steps before their first use
// through 4-byte cp.async copies, finished rows are stored as they leave), so
// many CTAs fit on an SM and hide each other's per-row latency.

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int RG, int D, int PF>
__global__ void batch_band_solve_win_kernel(const int32_t* __restrict__ node_off,
                                            const int32_t* __restrict__ bwv,
                                            const int64_t* __restrict__ band_off,
                                            const float* __restrict__ Lc, const float* __restrict__ Uc,
                                            float* __restrict__ V, int R, int64_t rs, int64_t cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ngroups = (R + RG - 1) / RG;
  const int t = blockIdx.x / ngroups;
  const int r0 = (blockIdx.x % ngroups) * RG;
  const int rg = min(RG, R - r0);
  const int base = node_off[t];
  const int n = node_off[t + 1] - base;
  const int bw = bwv[t];
  const int B = bw + 1;
  const int WB = bw + 1 + PF;  // window rows
  const float* lc = Lc + band_off[t];
  const float* uc = Uc + band_off[t];
  const int tid = threadIdx.x;
  float* win = reinterpret_cast<float*>(smem_raw);  // win[c * WB + row % WB]
  const int a = tid + 1;
  const bool act = a <= bw;
  const bool loader = tid < RG;  // thread c moves column c in and out
  const int c = tid;
  float* Vc = V + (int64_t)base * rs + (int64_t)(r0 + min(c, RG - 1)) * cs;  // row j at Vc[j rs]
  // ---- forward: rows [j, j + WB) in the window ----
  for (int i = tid; i < min(WB, n) * RG; i += blockDim.x) {
    const int cc = i / min(WB, n), row = i % min(WB, n);
    win[cc * WB + row] = cc < rg ? V[(int64_t)(base + row) * rs + (int64_t)(r0 + cc) * cs] : 0.f;
  }
  float pf[D], dg[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    pf[d] = (act && d < n && a <= n - 1 - d) ? lc[(size_t)d * B + a] : 0.f;
    dg[d] = (loader && d < n) ? lc[(size_t)d * B] : 0.f;
  }
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = j0 + d;
      if (j < n) {
        if (act && a <= n - 1 - j) {
          const float m = pf[d];
          const int dst = (j + a) % WB, src = j % WB;
#pragma unroll
          for (int q = 0; q < RG; ++q) win[q * WB + dst] -= m * win[q * WB + src];
        }
        const int jn = j + D;
        pf[d] = (act && jn < n && a <= n - 1 - jn) ? lc[(size_t)jn * B + a] : 0.f;
        __syncthreads();
        if (loader) {
          // row j is final: store y_j; bring row j + WB into its slot (first
          // used PF steps from now)
          const int slot = j % WB;
          if (c < rg) Vc[(int64_t)j * rs] = win[c * WB + slot] * dg[d];
          if (j + WB < n && c < rg) cp_async4(&win[c * WB + slot], Vc + (int64_t)(j + WB) * rs);
          cp_async_commit();
          dg[d] = jn < n ? lc[(size_t)jn * B] : 0.f;
          cp_async_wait<PF - 1>();
        }
        __syncthreads();
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // ---- backward: rows (j - WB, j] in the window, y read back ----
  for (int i = tid; i < min(WB, n) * RG; i += blockDim.x) {
    const int cc = i / min(WB, n), k = i % min(WB, n);
    const int row = n - 1 - k;
    win[cc * WB + row % WB] = cc < rg ? V[(int64_t)(base + row) * rs + (int64_t)(r0 + cc) * cs] : 0.f;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int j = n - 1 - d;
    pf[d] = (act && j >= 0 && a <= j) ? uc[(size_t)j * B + a] : 0.f;
    dg[d] = (loader && j >= 0) ? uc[(size_t)j * B] : 0.f;
  }
  __syncthreads();
  for (int j0 = n - 1; j0 >= 0; j0 -= D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = j0 - d;
      if (j >= 0) {
        if (act && a <= j) {
          const float m = pf[d];
          const int dst = (j - a) % WB, src = j % WB;
#pragma unroll
          for (int q = 0; q < RG; ++q) win[q * WB + dst] -= m * win[q * WB + src];
        }
        const int jn = j - D;
        pf[d] = (act && jn >= 0 && a <= jn) ? uc[(size_t)jn * B + a] : 0.f;
        __syncthreads();
        if (loader) {
          const int slot = j % WB;
          if (c < rg) Vc[(int64_t)j * rs] = win[c * WB + slot] * dg[d];
          if (j - WB >= 0 && c < rg) cp_async4(&win[c * WB + slot], Vc + (int64_t)(j - WB) * rs);
          cp_async_commit();
          dg[d] = jn >= 0 ? uc[(size_t)jn * B] : 0.f;
          cp_async_wait<PF - 1>();
        }
        __syncthreads();
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Blocked band solves: the rows of a tile in blocks of kBkNB, each block one
// dense product
// ---------------------------------------------------------------------------
//
// With L = L1 Dl^-1 (L1 unit lower, L1(j+a, j) = Lc[j][a]; Dl = diag(Lc[j][0]))
// the forward solve L y = v restricted to the block of rows [s, s + NB) is
//   y_blk = L_bb^-1 (v_blk - L[blk, win] y_win),   win = [s - W, s),
// W >= bw (only the last bw rows before the block reach it).  With
//   G_f = [ -L_bb^-1 L[blk, win] | L_bb^-1 ]            (NB x (W + NB))
// the block is y_blk = G_f [y_win; v_blk]: one product over the W + NB
// consecutive rows [s - W, s + NB).  Backward, with U = U1 Du^-1,
//   x_blk = U_bb^-1 (y_blk - U[blk, win'] x_win'),   win' = [s + NB, s + NB + W),
//   G_b = [ U_bb^-1 | -U_bb^-1 U[blk, win'] ]  over the rows [s, s + NB + W).
// G_f and G_b are formed once per factorisation in FP64 (substitutions local
// to each block on the band factors) and kept in FP32; a pass of the solve is
// then a chain of ceil(n / NB) small GEMMs instead of n dependent row steps.

constexpr int kBkNB = 64;                 // rows per block
constexpr int kBkRG = 64;                 // right-hand sides per CTA
constexpr int kBkS = 256;                 // ring rows; needs W + 2 NB <= kBkS
constexpr int kBkLd = kBkRG + 4;          // floats per ring row
constexpr int kBkStages = 4;              // G chunks (16 rows of G^T) in flight
constexpr int kBkThreads = 256;
constexpr int kBkMaxW = kBkS - 2 * kBkNB;  // widest window (bw <= 128)
constexpr int kBkLdx = 257;               // doubles per row of the set-up array
constexpr size_t kBkSmem = (size_t)(kBkS * kBkLd + kBkStages * 16 * kBkNB) * sizeof(float);
constexpr size_t kBkInvSmem = (size_t)kBkNB * kBkLdx * sizeof(double);

// One CTA per (block, pass).  Thread c takes column c of [-L[blk, win] | I]
// (forward) or [I | -U[blk, win']] (backward) through the block's own
// substitution with the pre-divided multipliers; the result times the
// block's diagonal factor is G, stored k-major (G[kk][i], kk the column) in
// FP32.  Backward blocks are stored in the order the solve visits them.
__global__ void __launch_bounds__(kBkThreads) blk_inverse_kernel(
    const int32_t* __restrict__ node_off, const int32_t* __restrict__ bwv,
    const int64_t* __restrict__ band_off, const int32_t* __restrict__ Wv,
    const int64_t* __restrict__ g_off, const int2* __restrict__ blk_list,
    const double* __restrict__ Lc, const double* __restrict__ Uc, float* __restrict__ Gf,
    float* __restrict__ Gb) {
  extern __shared__ double X[];  // X[i * kBkLdx + c]
  const int2 bk = blk_list[blockIdx.x];
  const int t = bk.x, k = bk.y;
  const bool fwd = blockIdx.y == 0;
  const int n = node_off[t + 1] - node_off[t];
  const int bw = bwv[t], B = bw + 1, W = Wv[t], K = W + kBkNB;
  const int nblk = (n + kBkNB - 1) / kBkNB;
  const int s = k * kBkNB;
  const int rows = min(kBkNB, n - s);
  const double* f = (fwd ? Lc : Uc) + band_off[t];
  const int c = threadIdx.x;
  if (c < K) {
    for (int i = 0; i < kBkNB; ++i) {
      double v = 0.0;
      if (i < rows) {
        if (fwd) {
          if (c >= W) {
            v = c - W == i ? 1.0 : 0.0;
          } else {
            const int w = s - W + c, a = s + i - w;  // -L(s + i, w)
            if (w >= 0 && a <= bw) v = -f[(size_t)w * B + a] / f[(size_t)w * B];
          }
        } else {
          if (c < kBkNB) {
            v = c == i ? 1.0 : 0.0;
          } else {
            const int w = s + c, b = w - (s + i);  // -U(s + i, w)
            if (w < n && b <= bw) v = -f[(size_t)w * B + b] / f[(size_t)w * B];
          }
        }
      }
      X[i * kBkLdx + c] = v;
    }
    if (fwd) {
      for (int j = 0; j < rows; ++j) {
        const double e = X[j * kBkLdx + c];
        if (e == 0.0) continue;
        const double* col = f + (size_t)(s + j) * B;
        const int m = min(bw, rows - 1 - j);
        for (int a = 1; a <= m; ++a) X[(j + a) * kBkLdx + c] -= col[a] * e;
      }
    } else {
      for (int j = rows - 1; j >= 0; --j) {
        const double e = X[j * kBkLdx + c];
        if (e == 0.0) continue;
        const double* col = f + (size_t)(s + j) * B;
        const int m = min(bw, j);
        for (int b = 1; b <= m; ++b) X[(j - b) * kBkLdx + c] -= col[b] * e;
      }
    }
  }
  __syncthreads();
  const int slot = fwd ? k : nblk - 1 - k;
  float* G = (fwd ? Gf : Gb) + g_off[t] + (size_t)slot * K * kBkNB;
  for (int e = threadIdx.x; e < K * kBkNB; e += blockDim.x) {
    const int kk = e / kBkNB, i = e % kBkNB;
    G[e] = i < rows ? (float)(f[(size_t)(s + i) * B] * X[i * kBkLdx + kk]) : 0.f;
  }
}

__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
// 16-byte copy (both addresses 16-byte aligned), zero-filled when !ok
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(ok ? 16 : 0)
               : "memory");
}
// 4-byte copy, zero-filled when !ok (the source is then not read)
__device__ __forceinline__ void cp_async4_zfill(void* smem, const void* gmem, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(ok ? 4 : 0)
               : "memory");
}

// One CTA per (tile, 64 right-hand sides): both passes.  Rows of the tile's
// column block live in a ring of kBkS rows (row g in slot g mod kBkS; rows
// outside [0, n) read as zero); the G^T of each block streams through
// kBkStages chunks of 16 rows by cp.async, and the input rows of the next
// block are fetched while the current one is multiplied.  Thread (ty, tx)
// accumulates rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3 of the block.
// V is addressed by strides (row-major FP32 work vectors: rs = R, cs = 1).
// Row-block moves between V and the ring: with whole rows of 16-byte groups,
// item e = tid + 256 m (m < 4) moves row e / 16, columns 4 (e % 16) .. + 3 as
// one 16-byte copy; otherwise 4-byte copies map lane l of warp w, step m, to
// row 8 (task & 7) + (l & 7), column 4 (task >> 3) + (l >> 3), task = w + 8 m.
// Both are conflict-free on the ring, and in both the same thread writes y in
// the forward pass and reads it back in the backward pass.
__global__ void __launch_bounds__(kBkThreads, 2) batch_band_solve_blk_kernel(
    const int32_t* __restrict__ node_off, const int32_t* __restrict__ Wv,
    const int64_t* __restrict__ g_off, const int32_t* __restrict__ order,
    const float* __restrict__ Gf, const float* __restrict__ Gb, float* __restrict__ V, int R,
    int64_t rs, int64_t cs) {
  extern __shared__ __align__(16) float bsm[];
  float* ring = bsm;
  float* gst = bsm + kBkS * kBkLd;
  const int ngroups = (R + kBkRG - 1) / kBkRG;
  const int t = order[blockIdx.x / ngroups];
  const int r0 = (blockIdx.x % ngroups) * kBkRG;
  const int rg = min(kBkRG, R - r0);
  const int base = node_off[t];
  const int n = node_off[t + 1] - base;
  const int W = Wv[t], KC = (W + kBkNB) / 16;
  const int nblk = (n + kBkNB - 1) / kBkNB;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  float* Vt = V + (int64_t)base * rs + (int64_t)r0 * cs;  // (row g, column c) at Vt[g rs + c cs]
  // row-major rows of whole 16-byte groups: 16-byte moves
  const bool vec4 = cs == 1 && (rs & 3) == 0;
  const int Q = nblk * KC;
  for (int pass = 0; pass < 2; ++pass) {
    const float* G = (pass == 0 ? Gf : Gb) + g_off[t];
    for (int i = tid; i < kBkS * kBkLd; i += kBkThreads) ring[i] = 0.f;
    __syncthreads();
    auto blk_start = [&](int b) { return (pass == 0 ? b : nblk - 1 - b) * kBkNB; };
    auto load_v = [&](int b) {
      if (b >= nblk) return;
      const int s = blk_start(b);
      if (vec4) {
        // row-major with whole 16-byte groups: item e = tid + 256 m is row
        // e / 16, columns 4 (e % 16) .. + 3 (a warp moves two 256-byte rows)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = tid + kBkThreads * m;
          const int g = s + (e >> 4), c = 4 * (e & 15);
          const bool ok = g < n && c < rg;
          cp_async16_zfill(&ring[(g & (kBkS - 1)) * kBkLd + c], ok ? Vt + (int64_t)g * rs + c : Vt, ok);
        }
        return;
      }
#pragma unroll 4
      for (int m = 0; m < 16; ++m) {
        const int task = warp + 8 * m;
        const int g = s + 8 * (task & 7) + (lane & 7);
        const int c = 4 * (task >> 3) + (lane >> 3);
        const bool ok = g < n && c < rg;
        cp_async4_zfill(&ring[(g & (kBkS - 1)) * kBkLd + c], ok ? Vt + (int64_t)g * rs + (int64_t)c * cs : Vt, ok);
      }
    };
    auto load_chunk = [&](int q) {
      if (q < Q)
        cp_async16_cg(&gst[(q % kBkStages) * 16 * kBkNB + tid * 4], G + (size_t)q * 16 * kBkNB + tid * 4);
    };
    load_v(0);
#pragma unroll
    for (int q = 0; q < kBkStages - 1; ++q) {
      load_chunk(q);
      cp_async_commit();
    }
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int q = 0; q < Q; ++q) {
      cp_async_wait<kBkStages - 2>();
      __syncthreads();
      const int b = q / KC, kc = q - b * KC;
      if (kc == 0) load_v(b + 1);
      load_chunk(q + kBkStages - 1);
      cp_async_commit();
      const int s = blk_start(b);
      const int row0 = (pass == 0 ? s - W : s) + 16 * kc;  // a multiple of 16: no wrap inside
      // the inverted diagonal block is triangular: a warp (rows 8 warp .. 8 warp
      // + 7) skips the chunks of it that are zero in all its rows
      const int j0 = pass == 0 ? 16 * kc - W : 16 * kc;  // first diagonal-block column
      const bool skip = pass == 0 ? (j0 >= 0 && j0 > 8 * warp + 7) : (j0 < kBkNB && j0 + 15 < 8 * warp);
      if (!skip) {
        const float* gq = gst + (q % kBkStages) * 16 * kBkNB + 4 * ty;
        const float* xq = ring + (row0 & (kBkS - 1)) * kBkLd + 4 * tx;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const float4 a = *reinterpret_cast<const float4*>(gq + kk * kBkNB);
          const float4 x = *reinterpret_cast<const float4*>(xq + kk * kBkLd);
          const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
        }
      }
      if (kc == KC - 1) {
        __syncthreads();  // every read of the block's input rows is done
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          *reinterpret_cast<float4*>(&ring[((s + 4 * ty + i) & (kBkS - 1)) * kBkLd + 4 * tx]) =
              make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        }
        __syncthreads();
        if (vec4) {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int e = tid + kBkThreads * m;
            const int g = s + (e >> 4), c = 4 * (e & 15);
            if (g < n && c < rg)
              *reinterpret_cast<float4*>(Vt + (int64_t)g * rs + c) =
                  *reinterpret_cast<const float4*>(&ring[(g & (kBkS - 1)) * kBkLd + c]);
          }
        } else {
#pragma unroll 4
          for (int m = 0; m < 16; ++m) {
            const int task = warp + 8 * m;
            const int g = s + 8 * (task & 7) + (lane & 7);
            const int c = 4 * (task >> 3) + (lane >> 3);
            if (g < n && c < rg) Vt[(int64_t)g * rs + (int64_t)c * cs] = ring[(g & (kBkS - 1)) * kBkLd + c];
          }
        }
      }
    }
    cp_async_wait<0>();
    __syncthreads();
  }
}

// Port-wise moves between [port][R] rows and the column-major [R][n] vectors
// go through a shared-memory tile of 32 ports x R: the [port][R] side is read
// or written along R, the vector side along the ports (whose nodes lie close
// together in the band order).

// c[s][r] = (2 W beta_s / d_s) x0[pos(s)][r]
template <class FT, class WT>
__global__ void __launch_bounds__(256) batch_const_kernel(const int32_t* __restrict__ port_pos,
                                                          const double* __restrict__ bout,
                                                          const FT* __restrict__ x0, WT* __restrict__ c,
                                                          int64_t nports, int R, int64_t n) {
  __shared__ WT tile[32][65];
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  const int ns = (int)(nports - s0 < 32 ? nports - s0 : 32);
  const int sl = threadIdx.x & 31;
  if (sl < ns) {
    const int64_t pos = port_pos[s0 + sl];
    const double bo = bout[s0 + sl];
    for (int r = threadIdx.x >> 5; r < R; r += 8) tile[sl][r] = (WT)(bo * (double)x0[(int64_t)r * n + pos]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ns * R; e += blockDim.x) c[s0 * R + e] = tile[e / R][e % R];
}

// V[pos(node)][r] += sum over the node's ports of beta_s w_in[s][r]
template <class FT, class WT>
__global__ void __launch_bounds__(256) batch_inject_kernel(const int32_t* __restrict__ port_pos,
                                                           const uint8_t* __restrict__ run,
                                                           const double* __restrict__ beta,
                                                           const WT* __restrict__ st, FT* __restrict__ V,
                                                           int64_t nports, int R, int64_t n) {
  __shared__ double tile[32][65];
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  const int ns = (int)(nports - s0 < 32 ? nports - s0 : 32);
  for (int e = threadIdx.x; e < ns * R; e += blockDim.x) {
    const int sl = e / R, r = e % R;
    const int64_t s = s0 + sl;
    const int nr = run[s];
    if (!nr) continue;
    double acc = 0.0;
    for (int q = 0; q < nr; ++q) acc += beta[s + q] * (double)st[(s + q) * 2 * R + r];
    tile[sl][r] = acc;
  }
  __syncthreads();
  const int sl = threadIdx.x & 31;
  if (sl < ns && run[s0 + sl]) {
    const int64_t pos = port_pos[s0 + sl];
    for (int r = threadIdx.x >> 5; r < R; r += 8) V[(int64_t)r * n + pos] += (FT)tile[sl][r];
  }
}

// ---------------------------------------------------------------------------
// the batched sweep
// ---------------------------------------------------------------------------

constexpr int kMB = 64;  // outputs per work item
constexpr int kKC = 16;  // inputs per chunk

// four consecutive shared-memory values (16-byte aligned) as vector reads
__device__ __forceinline__ void ld4_smem(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4_smem(const double* p, double (&o)[4]) {
  const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
  o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

// four consecutive values from global memory (16-byte aligned for FP32 and
// FP64, 8-byte for the 16-bit types), converted to the accumulate type
__device__ __forceinline__ void ld4_cvt(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4_cvt(const double* p, double (&o)[4]) {
  const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
  o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}
__device__ __forceinline__ void ld4_cvt(const __half* p, float (&o)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4_cvt(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
// four consecutive shared-memory values (16-byte aligned) as vector stores
__device__ __forceinline__ void st4_smem(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4_smem(double* p, const double (&v)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }

// Residual terms of the previous sweep for the node runs that start in
// [m0, m1) of the tile starting at port p0 (a run may reach past m1), per
// RHS: the square of each node's residual goes to rsq[run][r] (shared), and
// red[r] receives the column sums in a fixed order.  State layout:
// [port][2][R] = (w_in, w_out).
template <class WT, class RT>
__device__ void batch_residual(const int32_t* __restrict__ twin, const double2* __restrict__ kd,
                               const uint8_t* __restrict__ run, const WT* __restrict__ prev,
                               int p0, int m0, int m1, int R, RT (*rsq)[64], double* red) {
  // arithmetic in RT: FP32 for the low-precision sweeps (GB300's FP64 pipe is
  // narrow), FP64 for the FP64 sweep; kd = (g/W, d) of the line, the term is
  // d/2 [(S_s + S_t)/2 - (g/W)(S_s - S_t) - w_in(s) - w_in(t)], S = w_in + w_out
  for (int r = threadIdx.x; r < R; r += blockDim.x) red[r] = 0.0;
  // rows in slices of 32 node runs; the column sums add the slices in order
  for (int h0 = m0; h0 < m1; h0 += 32) {
    const int h1 = min(m1, h0 + 32);
    __syncthreads();
    for (int i = threadIdx.x; i < (h1 - h0) * R; i += blockDim.x) {
      const int sl = i / R;
      const int r = i % R;
      const int gs = p0 + h0 + sl;
      const int nr = run[gs];
      RT rsum = 0;
      for (int q = 0; q < nr; ++q) {
        const int ps = gs + q;
        const int tw = twin[ps];
        const RT wi_s = (RT)prev[(size_t)ps * 2 * R + r];
        const RT wo_s = (RT)prev[(size_t)ps * 2 * R + R + r];
        const RT wi_t = (RT)prev[(size_t)tw * 2 * R + r];
        const RT wo_t = (RT)prev[(size_t)tw * 2 * R + R + r];
        const double2 k2 = kd[ps];
        const RT Ss = wi_s + wo_s, St = wi_t + wo_t;
        rsum += (RT)0.5 * (RT)k2.y * ((RT)0.5 * (Ss + St) - (RT)k2.x * (Ss - St) - wi_s - wi_t);
      }
      rsq[sl][r] = rsum * rsum;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      RT a = 0;
      for (int sl = 0; sl < h1 - h0; ++sl) a += rsq[sl][r];
      red[r] += (double)a;
    }
  }
  __syncthreads();
}

// The per-item residual partials are summed in two fixed-order levels, so
// that no single CTA walks all items' rows one after another at the end of
// the sweep.  Work items are handed out by ticket and their partials stored
// by ticket ([ticket][R]); the tickets form groups of kBGrp, and the CTA
// that completes the last ticket of a group sums the group's rows into
// gsum[group][R] (gsum follows the nitems rows of the partials buffer; the
// group counters follow the BatchCtrl block).  The last CTA of the sweep
// then sums the group rows.  The order of every addition depends on the
// ticket numbers only, never on which CTA ran which item.
constexpr int kBGrp = 64;

// out[r] = sum of rows[0..nrows)[r]: G slices of consecutive rows, each with
// four interleaved accumulators, then the slices in order.  Called by every
// thread of the CTA; scr holds at least 256 doubles (shared).
__device__ void batch_ordered_sum(const double* rows, int nrows, int R, double* scr, double* out) {
  const int G = max(1, min((int)blockDim.x, 256) / R);
  const int t = threadIdx.x;
  if (t < G * R) {
    const int g = t / R, r = t % R;
    const int w0 = nrows * g / G, w1 = nrows * (g + 1) / G;
    scr[g * R + r] = ordered_sum_strided(rows + (size_t)w0 * R + r, w1 - w0, R);
  }
  __syncthreads();
  for (int r = t; r < R; r += blockDim.x) {
    double a = 0.0;
    for (int g = 0; g < G; ++g) a += scr[g * R + r];
    out[r] = a;
  }
  __syncthreads();
}

// After the partials of ticket `ticket` are stored and a CTA barrier: the
// group's counter, and the group sum by the CTA that completes the group.
__device__ void batch_item_done(BatchCtrl* __restrict__ ctrl, int ticket, int nitems, int R,
                                double* partials, double* scr) {
  __shared__ bool s_gl;
  unsigned* gcount = reinterpret_cast<unsigned*>(ctrl + 1);
  const int g = ticket / kBGrp;
  const int w0 = g * kBGrp, gn = min(kBGrp, nitems - w0);
  if (threadIdx.x == 0) {
    __threadfence();
    s_gl = atomicAdd(&gcount[g], 1u) == (unsigned)(gn - 1);
  }
  __syncthreads();
  if (!s_gl) return;
  __threadfence();
  batch_ordered_sum(partials + (size_t)w0 * R, gn, R, scr, partials + ((size_t)nitems + g) * R);
  if (threadIdx.x == 0) gcount[g] = 0u;  // ready for the next sweep
}

// Last-CTA reduction over the group sums per RHS and the convergence decision.
__device__ void batch_finish(BatchCtrl* __restrict__ ctrl, const double* __restrict__ partials,
                             int nitems, int R, const double* __restrict__ tol2,
                             double* __restrict__ hist, int hist_len, int k, double* scr) {
  __shared__ double worst;
  __shared__ int any_bad;
  __shared__ double fin[64];
  if (threadIdx.x == 0) {
    worst = 0.0;
    any_bad = 0;
  }
  batch_ordered_sum(partials + (size_t)nitems * R, (nitems + kBGrp - 1) / kBGrp, R, scr, fin);
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double tot = fin[r];
    if (!isfinite(tot)) atomicExch(&any_bad, 1);
    const double ratio = tot / tol2[r];
    // max over columns (atomicMax on the bit pattern of a non-negative double)
    atomicMax(reinterpret_cast<unsigned long long*>(&worst), __double_as_longlong(ratio));
    if (r == 0 && hist && k - 1 >= 1 && k - 1 <= hist_len) hist[k - 2] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int flag = 0;
    if (k > 1) {
      const int ks = k - 1;
      const double ratio = worst;
      if (ks == 1) ctrl->first_ratio = ratio;
      if (ks == 1 || ratio < 0.81 * ctrl->best_ratio) {
        ctrl->best_ratio = ratio;
        ctrl->best_k = ks;
      }
      if (any_bad || (ks > 1 && ratio > 1e12 * ctrl->first_ratio && ctrl->first_ratio > 0)) {
        flag = 3;
      } else if (ratio <= 1.0) {
        flag = 1;
        ctrl->conv_sweep = ks;
      } else if (ctrl->stall > 0 && ks - ctrl->best_k >= ctrl->stall) {
        flag = 4;
        ctrl->conv_sweep = ks;
      }
    }
    if (!flag && k >= ctrl->k_max) flag = 2;
    ctrl->counter = 0u;
    ctrl->work = 0u;
    ctrl->k = k + 1;
    __threadfence();
    ctrl->flag = flag;
  }
}

// CUDA-core version: 1024 / TM threads; thread (ty, tx) owns outputs
// m0 + TM ty .. +TM-1 and RHS 4 tx .. +3.  TT: stored T type; WT: wave type;
// AT: accumulate type.
template <class TT, class WT, class AT, int TM = 4>
__global__ void __launch_bounds__(1024 / TM) batch_sweep_kernel(
    const TT* __restrict__ T, const int64_t* __restrict__ T_off, const int32_t* __restrict__ T_ld,
    const int32_t* __restrict__ port_off, const int32_t* __restrict__ item_tile,
    const int32_t* __restrict__ item_m0, const int32_t* __restrict__ item_order, int nitems, const int32_t* __restrict__ twin,
    const double2* __restrict__ kd, const uint8_t* __restrict__ run, const WT* __restrict__ c,
    WT* __restrict__ state, int64_t nports, int R, BatchCtrl* __restrict__ ctrl,
    double* __restrict__ partials, const double* __restrict__ tol2, double* __restrict__ hist,
    int hist_len) {
  __shared__ __align__(16) AT Ts[2][kKC][kMB];  // double-buffered chunks
  __shared__ __align__(16) AT Ws[2][kKC][64];
  __shared__ double red[64];
  __shared__ AT rsq[32][64];
  __shared__ int s_k, s_flag;
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  if (tid < 64) red[tid] = 0.0;
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  // persistent: items of the longest-first work list until it is exhausted
  __shared__ int s_item;
  for (;;) {
  if (tid == 0) s_item = (int)atomicAdd(&ctrl->work, 1u);
  __syncthreads();
  if (s_item >= nitems) break;
  const int item = item_order[s_item];
  const int tile = item_tile[item];
  const int m0 = item_m0[item];
  const int p0 = port_off[tile];
  const int p = port_off[tile + 1] - p0;
  const int m1 = min(p, m0 + kMB);
  const int ld = T_ld[tile];
  const TT* Tb = T + T_off[tile];
  const WT* prev = state + (size_t)((k - 1) & 1) * nports * 2 * R;
  WT* cur = state + (size_t)(k & 1) * nports * 2 * R;
  if (k > 1) batch_residual<WT, AT>(twin, kd, run, prev, p0, m0, m1, R, rsq, red);
  constexpr int NT = 1024 / TM;
  static_assert(TM % 4 == 0 && TM * 4 * NT == kMB * 64, "thread tile");
  const int tx = tid % 16, ty = tid / 16;
  AT acc[TM][4];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  if (k > 1) {
    // acc += T(:, chunk)^T-block x W_in(chunk, :) from shared buffer b
    auto fma_chunk = [&](int b) {
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
        AT a[TM], bw[4];
#pragma unroll
        for (int i = 0; i < TM; i += 4)  // 16-byte (FP32) or 2 x 16-byte (FP64) reads
          ld4_smem(&Ts[b][kk][TM * ty + i], *reinterpret_cast<AT(*)[4]>(&a[i]));
        ld4_smem(&Ws[b][kk][4 * tx], bw);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bw[j];
      }
    };
    // Chunk loads are staged in registers one chunk ahead, so their latency
    // hides behind the FMAs; the twin rows that W_in is read through are
    // loaded one chunk earlier still, so that no load waits on another inside
    // the loop.  One barrier per chunk: buffer b is rewritten two chunks after
    // it was read, and every thread has passed the barrier of the chunk
    // between.  With R a multiple of 4 (and T's rows of whole 4-element
    // groups, as the layout pads them to 8) every load and shared store moves
    // a group of 4 consecutive outputs or right-hand sides: group g = tid +
    // e NT of a chunk is row g / 16, elements 4 (g % 16) .. + 3.
    const bool vec = (R & 3) == 0 && ((T_off[tile] | (int64_t)ld) & 3) == 0;
    if (vec) {
      constexpr int GT = kKC * 16 / NT;  // groups of T and of W_in per thread and chunk
      static_assert(GT * NT == kKC * 16, "chunk groups");
      AT tv[GT][4], wv[GT][4];
      int twv[GT];
      auto fetch_twin = [&](int t0) {
#pragma unroll
        for (int e = 0; e < GT; ++e) {
          const int t = t0 + (tid + e * NT) / 16;
          twv[e] = t < p ? twin[p0 + t] : 0;
        }
      };
      auto fetch = [&](int t0) {
#pragma unroll
        for (int e = 0; e < GT; ++e) {
          const int g = tid + e * NT;
          const int t = t0 + g / 16, c4 = 4 * (g % 16);
          if (t < p && m0 + c4 < m1) {
            ld4_cvt(Tb + (size_t)t * ld + m0 + c4, tv[e]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) tv[e][j] = AT(0);
          }
          if (t < p && c4 < R) {
            ld4_cvt(prev + (size_t)twv[e] * 2 * R + R + c4, wv[e]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) wv[e][j] = AT(0);
          }
        }
      };
      fetch_twin(0);
      fetch(0);
      fetch_twin(kKC);
      for (int t0 = 0, b = 0; t0 < p; t0 += kKC, b ^= 1) {
#pragma unroll
        for (int e = 0; e < GT; ++e) {
          const int g = tid + e * NT;
          st4_smem(&Ts[b][g / 16][4 * (g % 16)], tv[e]);
          st4_smem(&Ws[b][g / 16][4 * (g % 16)], wv[e]);
        }
        __syncthreads();
        if (t0 + kKC < p) {
          fetch(t0 + kKC);
          fetch_twin(t0 + 2 * kKC);
        }
        fma_chunk(b);
      }
    } else {
      // one element per load (NT threads x PT, PW elements of T and of W_in)
      constexpr int PT = kKC * kMB / NT, PW = kKC * 64 / NT;
      static_assert(PT * NT == kKC * kMB && PW * NT == kKC * 64, "chunk shape");
      AT tv[PT], wv[PW];
      int twv[PW];
      auto fetch_twin = [&](int t0) {
#pragma unroll
        for (int e = 0; e < PW; ++e) {
          const int t = t0 + (tid + e * NT) / 64;
          twv[e] = t < p ? twin[p0 + t] : 0;
        }
      };
      auto fetch = [&](int t0) {
#pragma unroll
        for (int e = 0; e < PT; ++e) {
          const int i = tid + e * NT;
          const int kk = i / kMB, mm = i % kMB;
          const int t = t0 + kk, s = m0 + mm;
          tv[e] = (t < p && s < m1) ? to_acc(Tb[(size_t)t * ld + s]) : AT(0);
        }
#pragma unroll
        for (int e = 0; e < PW; ++e) {
          const int i = tid + e * NT;
          const int kk = i / 64, r = i % 64;
          const int t = t0 + kk;
          wv[e] = (t < p && r < R) ? (AT)prev[(size_t)twv[e] * 2 * R + R + r] : AT(0);
        }
      };
      fetch_twin(0);
      fetch(0);
      fetch_twin(kKC);
      for (int t0 = 0, b = 0; t0 < p; t0 += kKC, b ^= 1) {
#pragma unroll
        for (int e = 0; e < PT; ++e) {
          const int i = tid + e * NT;
          Ts[b][i / kMB][i % kMB] = tv[e];
        }
#pragma unroll
        for (int e = 0; e < PW; ++e) {
          const int i = tid + e * NT;
          Ws[b][i / 64][i % 64] = wv[e];
        }
        __syncthreads();
        if (t0 + kKC < p) {
          fetch(t0 + kKC);
          fetch_twin(t0 + 2 * kKC);
        }
        fma_chunk(b);
      }
    }
  }
  // epilogue: w_out = acc + c, and this sweep's incident waves
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int s = m0 + TM * ty + i;
    if (s >= m1) continue;
    const size_t ps = (size_t)(p0 + s);
    const int tw = twin[p0 + s];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = 4 * tx + j;
      if (r >= R) continue;
      const WT wi = k > 1 ? prev[(size_t)tw * 2 * R + R + r] : WT(0);
      cur[ps * 2 * R + r] = wi;
      cur[ps * 2 * R + R + r] = (WT)(acc[i][j] + (AT)c[ps * R + r]);
    }
  }
  __syncthreads();
  for (int r = tid; r < R; r += blockDim.x) partials[(size_t)s_item * R + r] = k > 1 ? red[r] : 0.0;
  __syncthreads();
  batch_item_done(ctrl, s_item, nitems, R, partials, reinterpret_cast<double*>(&rsq[0][0]));
  }  // work list
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  batch_finish(ctrl, partials, nitems, R, tol2, hist, hist_len, k, reinterpret_cast<double*>(&rsq[0][0]));
}

// ---------------------------------------------------------------------------
// tensor-core version (BF16 T and incident waves, FP32 accumulate)
// ---------------------------------------------------------------------------
//
// CTA = 4 warps; warp w computes outputs m0 + 16 w .. +15 for all R (<= 64)
// RHS with mma.sync.m16n8k16 (A = T(s, t) read transposed from the stored
// T^T rows with ldmatrix.trans, B = W_in(t, r) read transposed from its
// row-major chunk).  Shared rows are padded by 8 elements (16 bytes) so the
// eight row addresses of each 8x8 ldmatrix fall in distinct bank groups.

constexpr int kAPad = kMB + 8;
constexpr int kBPad = 64 + 8;

__device__ __forceinline__ void ldsm_x4_trans(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                              const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) batch_sweep_mma_kernel(
    const __nv_bfloat16* __restrict__ T, const int64_t* __restrict__ T_off,
    const int32_t* __restrict__ T_ld, const int32_t* __restrict__ port_off,
    const int32_t* __restrict__ item_tile, const int32_t* __restrict__ item_m0, const int32_t* __restrict__ item_order, int nitems,
    const int32_t* __restrict__ twin, const double2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state,
    int64_t nports, int R, BatchCtrl* __restrict__ ctrl, double* __restrict__ partials,
    const double* __restrict__ tol2, double* __restrict__ hist, int hist_len) {
  constexpr int KC = 32;  // inputs per chunk (two k16 steps)
  __shared__ __align__(16) __nv_bfloat16 As[2][KC][kAPad];  // T^T chunk: [t][s], double-buffered
  __shared__ __align__(16) __nv_bfloat16 Bs[2][KC][kBPad];  // W_in chunk: [t][r]
  __shared__ double red[64];
  __shared__ float rsq[32][64];
  __shared__ int s_k, s_flag;
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  if (tid < 64) red[tid] = 0.0;
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  // persistent: items of the longest-first work list until it is exhausted
  __shared__ int s_item;
  for (;;) {
  if (tid == 0) s_item = (int)atomicAdd(&ctrl->work, 1u);
  __syncthreads();
  if (s_item >= nitems) break;
  const int item = item_order[s_item];
  const int tile = item_tile[item];
  const int m0 = item_m0[item];
  const int p0 = port_off[tile];
  const int p = port_off[tile + 1] - p0;
  const int m1 = min(p, m0 + kMB);
  const int ld = T_ld[tile];
  const __nv_bfloat16* Tb = T + T_off[tile];
  const float* prev = state + (size_t)((k - 1) & 1) * nports * 2 * R;
  float* cur = state + (size_t)(k & 1) * nports * 2 * R;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
  const int ntiles = (R + 7) / 8;
  // per thread: 2 16-byte pieces of the T chunk and 4 float4 of the wave chunk
  uint4 ra[2];
  float4 rb[4];
  auto load_chunk = [&](int t0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = tid + q * 128;
      const int kk = i / 8, piece = i % 8;
      const int t = t0 + kk, s = m0 + piece * 8;
      ra[q] = (t < p && s < m1) ? __ldcs(reinterpret_cast<const uint4*>(Tb + (size_t)t * ld + s))
                                : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = tid + q * 128;
      const int kk = i / 16, r = (i % 16) * 4;
      const int t = t0 + kk;
      rb[q] = (t < p && r < R)
                  ? *reinterpret_cast<const float4*>(prev + (size_t)twin[p0 + t] * 2 * R + R + r)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store_chunk = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = tid + q * 128;
      *reinterpret_cast<uint4*>(&As[buf][i / 8][(i % 8) * 8]) = ra[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = tid + q * 128;
      const int kk = i / 16, r = (i % 16) * 4;
      *reinterpret_cast<__nv_bfloat162*>(&Bs[buf][kk][r]) = __floats2bfloat162_rn(rb[q].x, rb[q].y);
      *reinterpret_cast<__nv_bfloat162*>(&Bs[buf][kk][r + 2]) = __floats2bfloat162_rn(rb[q].z, rb[q].w);
    }
  };
  if (k > 1) {
    load_chunk(0);  // in flight during the residual of sweep k-1
    batch_residual<float, float>(twin, kd, run, prev, p0, m0, m1, R, rsq, red);
    int buf = 0;
    for (int t0 = 0; t0 < p; t0 += KC, buf ^= 1) {
      store_chunk(buf);
      __syncthreads();
      if (t0 + KC < p) load_chunk(t0 + KC);  // next chunk streams while this one multiplies
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        uint32_t a0, a1, a2, a3;
        {
          const int mat = lane >> 3, row = lane & 7;
          const int kk = ks * 16 + row + ((mat >> 1) << 3);  // matrices 2,3: inputs 8..15
          const int mm = warp * 16 + ((mat & 1) << 3);       // matrices 1,3: outputs 8..15
          ldsm_x4_trans(a0, a1, a2, a3, &As[buf][kk][mm]);
        }
#pragma unroll
        for (int np = 0; np < 4; ++np) {  // pairs of 8-wide RHS tiles
          if (2 * np >= ntiles) break;
          uint32_t b0, b1, b2, b3;
          const int mat = lane >> 3, row = lane & 7;
          const int kk = ks * 16 + row + ((mat & 1) << 3);  // matrices 1,3: inputs 8..15
          const int nn = np * 16 + ((mat >> 1) << 3);       // matrices 2,3: next RHS tile
          ldsm_x4_trans(b0, b1, b2, b3, &Bs[buf][kk][nn]);
          mma_bf16(acc[2 * np], a0, a1, a2, a3, b0, b1);
          mma_bf16(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
        }
      }
    }
  }
  // epilogue: fragment element e of tile nt sits at output row
  // warp*16 + lane/4 (+8 for e >= 2) and RHS column nt*8 + 2*(lane%4) + (e&1)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    if (nt >= ntiles) break;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int s = m0 + warp * 16 + (lane >> 2) + ((e >> 1) << 3);
      const int r = nt * 8 + 2 * (lane & 3) + (e & 1);
      if (s < m1 && r < R) {
        const size_t ps = (size_t)(p0 + s);
        const float wi = k > 1 ? prev[(size_t)twin[p0 + s] * 2 * R + R + r] : 0.f;
        cur[ps * 2 * R + r] = wi;
        cur[ps * 2 * R + R + r] = acc[nt][e] + c[ps * R + r];
      }
    }
  }
  __syncthreads();
  for (int r = tid; r < R; r += blockDim.x) partials[(size_t)s_item * R + r] = k > 1 ? red[r] : 0.0;
  __syncthreads();
  batch_item_done(ctrl, s_item, nitems, R, partials, reinterpret_cast<double*>(&rsq[0][0]));
  }  // work list
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  batch_finish(ctrl, partials, nitems, R, tol2, hist, hist_len, k, reinterpret_cast<double*>(&rsq[0][0]));
}

// ---------------------------------------------------------------------------
// tcgen05 version (BF16 T and incident waves, FP32 accumulators in TMEM)
// ---------------------------------------------------------------------------
//
// W_out(P) = T_P W_in(P) + C_P for up to 64 right-hand sides is a dense
// contraction (Eq. 11 with many right-hand sides): M = the box's output ports,
// K = its input ports, N = 64 columns.  A work item is a box and up to four
// 128-row M tiles (512 outputs: 4 accumulators of 128 lanes x 64 FP32
// columns, 256 TMEM columns); items run longest first from a work list over
// persistent CTAs of 128 threads, two per SM.
//   * A: T_P in 128 x 64 BF16 tiles prepared at factor time in the UMMA
//     canonical K-major layout without swizzle (8 x 8 core matrices of 128
//     bytes, the eight K groups of a row group adjacent: LBO = 128 B, SBO =
//     1 KB), each item's tiles contiguous in consumption order (input chunk,
//     then M tile), so one 16 KB bulk copy fills a stage of a 4-stage ring
//     (mbarriers with transaction counts), issued three tiles ahead by thread
//     0, which also issues the MMAs;
//   * B: the incident waves of a 64-input chunk, gathered from the twins'
//     outgoing waves of the previous sweep (FP32) by all threads, rounded to
//     BF16 and written in the same canonical layout (double-buffered; a
//     buffer is rewritten once the MMAs that read it have committed);
//   * per chunk and M tile, four tcgen05.mma (M = 128, N = 64, K = 16) add
//     into the tile's TMEM accumulator; tcgen05.commit frees the A stage and,
//     after the chunk's last tile, the B buffer;
//   * epilogue: each warp reads its 32 TMEM lanes (tcgen05.ld 32x32b), adds
//     C and writes w_out; the residual terms of the previous sweep and the
//     decision are those of the other batched kernels.
// Every mbarrier wait is bounded (kTcPolls); a wait that runs out sets flag 5
// (VTM_ETIMEOUT), and the CTA waits (bounded) for its copies and MMAs in
// flight, frees its TMEM columns and leaves.
constexpr int kTcM = 128;                            // rows per MMA tile
constexpr int kTcK = 64;                             // inputs per chunk
constexpr int kTcG = 4;                              // M tiles per work item
constexpr int kTcS = 3;                              // A stages
constexpr uint32_t kTcTileBytes = kTcM * kTcK * 2;   // 16 KB
constexpr uint32_t kTcBBytes = 64 * kTcK * 2;        // 8 KB
constexpr uint32_t kTcCols = 64 * kTcG;              // TMEM columns per CTA
constexpr uint32_t kTcPolls = 1u << 24;
constexpr int kTcThreads = 256;                      // 8 warps: two per TMEM lane quarter
constexpr int kTcLd = 68;                            // FP32 staging row stride (conflict-free columns)
constexpr size_t kTcSmem = kTcS * (size_t)kTcTileBytes + 2 * (size_t)kTcBBytes + 2 * (size_t)kTcK * kTcLd * 4 + 1024;

// smem matrix descriptor: canonical K-major, no swizzle (LBO = 128 B between
// the two K core matrices of a K = 16 step, SBO = 1 KB between 8-row groups)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
  return d;
}
// instruction descriptor: F32 accumulate, BF16 A and B, both K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void cp_async16_tc(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// 16 FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 2) batch_sweep_tc_kernel(
    const __nv_bfloat16* __restrict__ Ttc, const int4* __restrict__ items, const int64_t* __restrict__ item_off,
    const int32_t* __restrict__ item_order, int nitems, const int32_t* __restrict__ port_off,
    const int32_t* __restrict__ twin, const double2* __restrict__ kd, const uint8_t* __restrict__ run,
    const float* __restrict__ c, float* __restrict__ state, int64_t nports, int R,
    BatchCtrl* __restrict__ ctrl, double* __restrict__ partials, const double* __restrict__ tol2,
    double* __restrict__ hist, int hist_len) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  // 1 KB alignment of the stage buffers (canonical layouts need 16 B; the
  // descriptors' base-offset field stays 0)
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  unsigned char* As = base;
  unsigned char* Bs = As + kTcS * kTcTileBytes;
  float* Sg = reinterpret_cast<float*>(Bs + 2 * kTcBBytes);  // 2 x 64 staging rows
  const bool vecR = (R & 3) == 0;
  __shared__ uint64_t full[kTcS], empty[kTcS], bfull[2], bdone[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_k, s_flag, s_item, s_abort;
  __shared__ bool s_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
    s_abort = 0;
    for (int i = 0; i < kTcS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&bdone[0], 1);
    mbar_init(&bdone[1], 1);
    mbar_init(&bfull[0], kTcThreads - 64);
    mbar_init(&bfull[1], kTcThreads - 64);
    fence_mbar_init();
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  // counters of this CTA over its items: A tiles issued (thread 0) and chunks
  uint32_t q_issued = 0, q_base = 0, cg = 0;
  auto abort_wait = [&]() {
    atomicCAS(&ctrl->flag, 0, 5);
    s_abort = 1;
  };
  // thread 0 (the producer): tile gq of this CTA's sequence into its stage
  // (after the MMAs that read the stage's previous tile have committed)
  auto issue_tile = [&](uint32_t gq, const __nv_bfloat16* src) -> bool {
    const uint32_t st = gq % kTcS;
    if (gq >= kTcS && !mbar_wait_bounded(&empty[st], ((gq / kTcS) - 1) & 1, kTcPolls)) return false;
    mbar_arrive_expect_tx(&full[st], kTcTileBytes);
    bulk_copy_g2s(As + st * kTcTileBytes, src, kTcTileBytes, &full[st]);
    q_issued = gq + 1;
    return true;
  };
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(&ctrl->work, 1u);
    __syncthreads();
    if (s_item >= nitems || s_abort) break;
    const int item = item_order[s_item];
    const int4 it = items[item];
    const int tile = it.x, m0 = it.y, nmt = it.z, nkc = it.w;
    const int p0 = port_off[tile];
    const int p = port_off[tile + 1] - p0;
    const int m1 = min(p, m0 + nmt * kTcM);
    const __nv_bfloat16* Ab = Ttc + item_off[item];
    const float* prev = state + (size_t)((k - 1) & 1) * nports * 2 * R;
    float* cur = state + (size_t)(k & 1) * nports * 2 * R;
    const int ntot = nmt * nkc;
    if (k > 1) {
      // Warp-specialised main loop: warp 0 (lane 0) streams the item's A
      // tiles into the ring as stages free up; warp 1 (lane 0) issues the
      // MMAs as tiles and B chunks become ready; warps 2-7 gather the B
      // chunks.  No CTA barrier inside: mbarriers order everything (full /
      // empty per A stage, bfull / bdone per B buffer), and every role runs
      // its fixed number of steps, skipping its waits after an abort.
      if (warp == 0) {
        if (lane == 0)
          for (int q = 0; q < ntot; ++q)
            if (!s_abort && !issue_tile(q_base + q, Ab + (size_t)q * (kTcTileBytes / 2))) abort_wait();
      } else if (warp == 1) {
        if (lane == 0) {
          for (int kc = 0; kc < nkc; ++kc) {
            const uint32_t c2 = cg + kc, buf = c2 & 1;
            if (!s_abort && !mbar_wait_bounded(&bfull[buf], (c2 >> 1) & 1, kTcPolls)) abort_wait();
            tc_fence_after();
            const uint32_t b0 = smem_u32(Bs + buf * kTcBBytes);
            for (int mt = 0; mt < nmt; ++mt) {
              const uint32_t gq = q_base + kc * nmt + mt, st = gq % kTcS;
              if (s_abort || !mbar_wait_bounded(&full[st], (gq / kTcS) & 1, kTcPolls)) {
                abort_wait();
                break;
              }
              tc_fence_after();
              const uint32_t a0 = smem_u32(As + st * kTcTileBytes);
#pragma unroll
              for (int ks = 0; ks < kTcK / 16; ++ks)
                tc_mma(tmem + mt * 64, tc_desc(a0 + 256 * ks), tc_desc(b0 + 256 * ks), (kc > 0 || ks > 0) ? 1u : 0u);
              tc_commit(&empty[st]);
            }
            tc_commit(&bdone[buf]);
          }
        }
      } else {
        // B builders: the 64 twin rows of chunk j (their outgoing waves, 64
        // FP32 columns) are copied into FP32 staging rows (cp.async, one
        // chunk ahead, double-buffered; plain loads when R is not a multiple
        // of 4), then rounded to BF16 into the canonical B layout
        const int bt = tid - 64;  // builder thread 0..191
        constexpr int NB = kTcThreads - 64;
        auto stage_rows = [&](int j) {
          float* stg = Sg + (j & 1) * kTcK * kTcLd;
          for (int e = bt; e < kTcK * 16; e += NB) {
            const int r = e >> 4, seg = e & 15;
            const int t = j * kTcK + r;
            const int tw = t < p ? twin[p0 + t] : -1;
            float* dst = stg + r * kTcLd + seg * 4;
            if (tw >= 0 && vecR && seg * 4 < R) {
              cp_async16_tc(dst, prev + (size_t)tw * 2 * R + R + seg * 4);
            } else if (tw >= 0 && !vecR) {
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) dst[q4] = seg * 4 + q4 < R ? prev[(size_t)tw * 2 * R + R + seg * 4 + q4] : 0.f;
            } else {
              *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
        };
        stage_rows(0);
        for (int kc = 0; kc < nkc; ++kc) {
          const uint32_t c2 = cg + kc, buf = c2 & 1;
          unsigned char* Bb = Bs + buf * kTcBBytes;
          asm volatile("cp.async.wait_group 0;" ::: "memory");  // this thread's rows of chunk kc
          // every builder's rows of chunk kc have landed, and every builder
          // has converted chunk kc - 1 (its staging rows may be refilled)
          asm volatile("bar.sync 1, %0;" ::"r"(NB) : "memory");
          if (kc + 1 < nkc) stage_rows(kc + 1);
          // the MMAs of chunk c2 - 2 read this B buffer
          if (c2 >= 2 && !s_abort && !mbar_wait_bounded(&bdone[buf], ((c2 - 2) >> 1) & 1, kTcPolls)) abort_wait();
          const float* stg = Sg + (kc & 1) * kTcK * kTcLd;
          // 64 columns x 8 input groups: eight inputs of one column per 16 bytes
          for (int pi = bt; pi < 64 * 8; pi += NB) {
            const int n = pi & 63, kg = pi >> 6;
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(stg[(kg * 8 + 2 * e) * kTcLd + n],
                                                             stg[(kg * 8 + 2 * e + 1) * kTcLd + n]);
              w[e] = *reinterpret_cast<const uint32_t*>(&h);
            }
            *reinterpret_cast<uint4*>(Bb + ((n >> 3) * 8 + kg) * 128 + (n & 7) * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
          }
          fence_proxy_async_smem();  // the generic-proxy writes of B, before the MMAs read them
          mbar_arrive(&bfull[buf]);
        }
      }
      cg += nkc;
      q_base += ntot;
      // every MMA of the item has completed once its last chunk's commit has
      if (!s_abort && !mbar_wait_bounded(&bdone[(cg - 1) & 1], ((cg - 1) >> 1) & 1, kTcPolls)) abort_wait();
      tc_fence_after();
    }
    __syncthreads();
    if (s_abort) break;
    // Epilogue, one M tile at a time: the accumulators go through shared
    // memory (the idle A ring: 128 rows of 64 floats, row stride 68) so that
    // the global accesses run along the right-hand sides of a port (16
    // threads x 4 columns per row, 8 rows per pass): w_out = T W_in + c, this
    // sweep's w_in, and the residual terms of the previous sweep for the node
    // runs that start in the item (each run's terms summed in port order, then
    // squared), the same arithmetic as batch_residual.
    float* tr = reinterpret_cast<float*>(As);
    constexpr int kTrLd = 68;
    constexpr int kRowSlots = kTcThreads / 16;
    const int cq = tid & 15, rq = tid >> 4;  // column group, row slot
    float sq[4] = {0.f, 0.f, 0.f, 0.f};
    const bool vec = (R & 3) == 0;
    const int quarter = warp & 3, half = warp >> 2;  // TMEM lanes 32 quarter.., columns 32 half..
    for (int mt = 0; mt < nmt; ++mt) {
      if (k > 1) {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          float v[16];
          const int col = half * 32 + cc * 16;
          tc_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + mt * 64 + col, v);
          float* dst = tr + (32 * quarter + lane) * kTrLd + col;
#pragma unroll
          for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
      // the tile's port tables (twin, node run, g/W, d/2) into the idle B buffers
      int* mtw = reinterpret_cast<int*>(Bs);
      int* mrn = mtw + kTcM;
      float2* mkd = reinterpret_cast<float2*>(mrn + kTcM);
      float* tm = Sg;  // residual term of every port of the tile (rows of 68)
      if (tid < kTcM) {
        const int s = m0 + mt * kTcM + tid;
        int tw = 0, nr = 0;
        float2 kk = make_float2(0.f, 0.f);
        if (s < m1) {
          const size_t ps = (size_t)(p0 + s);
          tw = twin[ps];
          nr = run[ps];
          const double2 k2 = kd[ps];
          kk = make_float2((float)k2.x, 0.5f * (float)k2.y);
        }
        mtw[tid] = tw;
        mrn[tid] = nr;
        mkd[tid] = kk;
      }
      __syncthreads();
      auto load4 = [&](const float* src, int r0, float (&o)[4]) {
        if (vec) {
          const float4 f = *reinterpret_cast<const float4*>(src);
          o[0] = f.x; o[1] = f.y; o[2] = f.z; o[3] = f.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) o[j] = r0 + j < R ? src[j] : 0.f;
        }
      };
      auto store4 = [&](float* dst, int r0, const float (&o)[4]) {
        if (vec) {
          *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (r0 + j < R) dst[j] = o[j];
        }
      };
      // residual term of port pq (twin tq) for columns r0..+3: the arithmetic
      // of batch_residual
      auto term4 = [&](const float (&wis)[4], const float (&wos)[4], const float (&wit)[4],
                       const float (&wot)[4], float2 kq, float (&t)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float Ss = wis[j] + wos[j], St = wit[j] + wot[j];
          t[j] = kq.y * (0.5f * (Ss + St) - kq.x * (Ss - St) - wis[j] - wit[j]);
        }
      };
      const int r0 = 4 * cq;
      // outputs and every port's residual term: two rows of this thread at a
      // time, all their loads issued together
      constexpr int kRows = kTcM / kRowSlots;  // rows per thread and tile
      for (int i0 = 0; i0 < kRows; i0 += 2) {
        float cv[2][4], wt[2][4], wis[2][4], wos[2][4], wit[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int row = rq + kRowSlots * (i0 + u);
          const int s = m0 + mt * kTcM + row;
          const size_t ps = (size_t)(p0 + (s < m1 ? s : 0));
#pragma unroll
          for (int j = 0; j < 4; ++j) cv[u][j] = wt[u][j] = wis[u][j] = wos[u][j] = wit[u][j] = 0.f;
          if (s < m1 && r0 < R) {
            load4(c + ps * R + r0, r0, cv[u]);
            if (k > 1) {
              const size_t tw = (size_t)mtw[row];
              load4(prev + tw * 2 * R + R + r0, r0, wt[u]);
              load4(prev + ps * 2 * R + r0, r0, wis[u]);
              load4(prev + ps * 2 * R + R + r0, r0, wos[u]);
              load4(prev + tw * 2 * R + r0, r0, wit[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int row = rq + kRowSlots * (i0 + u);
          const int s = m0 + mt * kTcM + row;
          if (s < m1 && r0 < R) {
            const size_t ps = (size_t)(p0 + s);
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = (k > 1 ? tr[row * kTrLd + r0 + j] : 0.f) + cv[u][j];
            store4(cur + ps * 2 * R + r0, r0, wt[u]);
            store4(cur + ps * 2 * R + R + r0, r0, o);
            if (k > 1) {
              float t[4];
              term4(wis[u], wos[u], wit[u], wt[u], mkd[row], t);
#pragma unroll
              for (int j = 0; j < 4; ++j) tm[row * kTrLd + r0 + j] = t[j];
            }
          }
        }
      }
      __syncthreads();
      // the nodes whose runs of ports start in the tile: each run's terms
      // summed in port order, then squared (ports past the tile's last row
      // come from global memory)
      if (k > 1 && r0 < R) {
        for (int i = 0; i < kRows; ++i) {
          const int row = rq + kRowSlots * i;
          const int s = m0 + mt * kTcM + row;
          if (s >= m1) break;
          const int nr = mrn[row];
          if (!nr) continue;
          float rs[4] = {0.f, 0.f, 0.f, 0.f};
          for (int qq = 0; qq < nr; ++qq) {
            float t[4];
            const int rowq = row + qq;
            if (rowq < kTcM) {
#pragma unroll
              for (int j = 0; j < 4; ++j) t[j] = tm[rowq * kTrLd + r0 + j];
            } else {
              const size_t pq = (size_t)(p0 + s + qq);
              const size_t tq = (size_t)twin[pq];
              const double2 k2 = kd[pq];
              float a1[4], a2[4], a3[4], a4[4];
              load4(prev + pq * 2 * R + r0, r0, a1);
              load4(prev + pq * 2 * R + R + r0, r0, a2);
              load4(prev + tq * 2 * R + r0, r0, a3);
              load4(prev + tq * 2 * R + R + r0, r0, a4);
              term4(a1, a2, a3, a4, make_float2((float)k2.x, 0.5f * (float)k2.y), t);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) rs[j] += t[j];
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) sq[j] += rs[j] * rs[j];
        }
      }
      __syncthreads();  // before the next tile's accumulators overwrite the staging rows
    }
    tc_fence_before();  // these TMEM reads precede the next item's MMAs
    // the item's squared residual per column: the row slots in order (lanes
    // l and l + 16 of a warp, then the warps)
    double* red8 = reinterpret_cast<double*>(tr);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float o16 = __shfl_xor_sync(0xffffffffu, sq[j], 16);
      if (lane < 16) red8[warp * 64 + 4 * cq + j] = (double)sq[j] + (double)o16;
    }
    __syncthreads();
    for (int r = tid; r < R; r += blockDim.x) {
      double t = 0.0;
      if (k > 1)
        for (int w8 = 0; w8 < kTcThreads / 32; ++w8) t += red8[w8 * 64 + r];
      partials[(size_t)s_item * R + r] = t;
    }
    __syncthreads();
    // the staging rows are free until the next item's epilogue
    batch_item_done(ctrl, s_item, nitems, R, partials, reinterpret_cast<double*>(Sg));
  }  // work list
  if (s_abort && warp == 0 && lane == 0) {
    // copies in flight land before the CTA releases its shared memory (bounded)
    for (uint32_t gq = (q_issued > kTcS ? q_issued - kTcS : 0); gq < q_issued; ++gq)
      mbar_wait_bounded(&full[gq % kTcS], (gq / kTcS) & 1, kTcPolls);
  }
  if (s_abort && warp == 1 && lane == 0) {
    // and the MMAs issued complete before it releases its TMEM (bounded)
    tc_commit(&bdone[cg & 1]);
    mbar_wait_bounded(&bdone[cg & 1], (cg >> 1) & 1, kTcPolls);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  if (s_abort) return;
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  batch_finish(ctrl, partials, nitems, R, tol2, hist, hist_len, k, reinterpret_cast<double*>(Sg));
}

// T_P of every work item in the tcgen05 tile layout: tile q = kc * nmt + mt
// of the item holds T_P(s, t) for s = m0 + 128 mt + m, t = 64 kc + kk at core
// matrix (m / 8, kk / 8), row m % 8, element kk % 8 (BF16, zero outside p);
// T_P(s, t) is element t ld + s of the tile's T^T block.
__global__ void pack_tc_kernel(const double* __restrict__ T64, const int64_t* __restrict__ T_off,
                               const int32_t* __restrict__ T_ld, const int32_t* __restrict__ port_off,
                               const int4* __restrict__ items, const int64_t* __restrict__ item_off,
                               __nv_bfloat16* __restrict__ out) {
  const int4 it = items[blockIdx.x];
  const int tile = it.x, m0 = it.y, nmt = it.z, nkc = it.w;
  const int p = port_off[tile + 1] - port_off[tile];
  const int ld = T_ld[tile];
  const double* Tt = T64 + T_off[tile];
  __nv_bfloat16* o = out + item_off[blockIdx.x];
  const int64_t nel = (int64_t)nmt * nkc * kTcM * kTcK;
  for (int64_t i = threadIdx.x; i < nel; i += blockDim.x) {
    const int q = (int)(i / (kTcM * kTcK)), e = (int)(i % (kTcM * kTcK));
    const int kc = q / nmt, mt = q % nmt;
    const int core = e / 64, w = e % 64;
    const int m = (core / 8) * 8 + w / 8, kk = (core % 8) * 8 + w % 8;
    const int s = m0 + mt * kTcM + m, t = kc * kTcK + kk;
    const double v = (s < p && t < p) ? Tt[(size_t)t * ld + s] : 0.0;
    o[i] = __float2bfloat16_rn((float)v);
  }
}

// ---------------------------------------------------------------------------
// host driver for a batch of right-hand sides
// ---------------------------------------------------------------------------

static int grid_n(int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 16));
}

static vtm_status batch_band_solve_win(vtm_plan_s* P, float* V, int R, const float* Lc,
                                       const float* Uc) {
  constexpr int RG = 16, D = 8, PF = 8;
  const int ngroups = (R + RG - 1) / RG;
  const int threads = std::max(32, (std::max(P->max_bw, RG) + 31) / 32 * 32);
  const size_t smem = (size_t)(P->max_bw + 1 + PF) * RG * sizeof(float);
  if (threads > 1024 || smem > 200 * 1024) {
    set_detail("batched solve: band too wide for the windowed batched band solve");
    return VTM_EINVAL;
  }
  if (smem > 48 * 1024)
    VTM_CUDA_TRY(cudaFuncSetAttribute(batch_band_solve_win_kernel<RG, D, PF>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  batch_band_solve_win_kernel<RG, D, PF><<<P->nparts * ngroups, threads, smem, P->stream>>>(
      P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(), Lc,
      Uc, V, R, (int64_t)R, (int64_t)1);
  P->launch_count++;
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

// The blocked solve's tables and G_f / G_b, formed from the FP64 band
// factors (once per factorisation).
static vtm_status blk_prepare(vtm_plan_s* P) {
  if (P->bk_ready) return VTM_OK;
  cudaStream_t s = P->stream;
  std::vector<int32_t> W(P->nparts), order(P->nparts);
  std::vector<int64_t> goff(P->nparts), cost(P->nparts);
  std::vector<int2> blks;
  int64_t o = 0;
  for (int32_t t = 0; t < P->nparts; ++t) {
    const int n = P->node_off[t + 1] - P->node_off[t];
    const int nblk = (n + kBkNB - 1) / kBkNB;
    W[t] = (P->bw[t] + 15) / 16 * 16;
    goff[t] = o;
    cost[t] = (int64_t)nblk * (W[t] + kBkNB);
    for (int k = 0; k < nblk; ++k) blks.push_back(make_int2(t, k));
    o += (int64_t)nblk * (W[t] + kBkNB) * kBkNB;
    order[t] = t;
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  VTM_TRY(upload(P->d_bk_W, W, s));
  VTM_TRY(upload(P->d_bk_goff, goff, s));
  VTM_TRY(upload(P->d_bk_order, order, s));
  VTM_TRY(upload(P->d_bk_blk, blks, s));
  VTM_TRY(dev_alloc(P->d_bk_Gf, (size_t)std::max<int64_t>(o, 16) * sizeof(float)));
  VTM_TRY(dev_alloc(P->d_bk_Gb, (size_t)std::max<int64_t>(o, 16) * sizeof(float)));
  if (!blks.empty()) {
    VTM_CUDA_TRY(cudaFuncSetAttribute(blk_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kBkInvSmem));
    blk_inverse_kernel<<<dim3((unsigned)blks.size(), 2), kBkThreads, kBkInvSmem, s>>>(
        P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(),
        P->d_bk_W.as<int32_t>(), P->d_bk_goff.as<int64_t>(), P->d_bk_blk.as<int2>(),
        P->d_Lc.as<double>(), P->d_Uc.as<double>(), P->d_bk_Gf.as<float>(), P->d_bk_Gb.as<float>());
    P->launch_count++;
    VTM_CUDA_TRY(cudaGetLastError());
  }
  P->bk_ready = true;
  return VTM_OK;
}

static vtm_status batch_band_solve_blk(vtm_plan_s* P, float* V, int R) {
  if (P->max_bw > kBkMaxW) {
    set_detail("batched solve: the blocked band solve takes half bandwidths up to 128");
    return VTM_EINVAL;
  }
  VTM_TRY(blk_prepare(P));
  const int ngroups = (R + kBkRG - 1) / kBkRG;
  VTM_CUDA_TRY(cudaFuncSetAttribute(batch_band_solve_blk_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBkSmem));
  batch_band_solve_blk_kernel<<<P->nparts * ngroups, kBkThreads, kBkSmem, P->stream>>>(
      P->tabs.node_off.as<int32_t>(), P->d_bk_W.as<int32_t>(), P->d_bk_goff.as<int64_t>(),
      P->d_bk_order.as<int32_t>(), P->d_bk_Gf.as<float>(), P->d_bk_Gb.as<float>(), V, R, (int64_t)R,
      (int64_t)1);
  P->launch_count++;
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

template <class FT>
static vtm_status batch_band_solve(vtm_plan_s* P, FT* V, int R, const FT* Lc, const FT* Uc) {
  if constexpr (sizeof(FT) == 4) {
    const int mode = P->opts.batch_solve;
    if (mode == 3 || (mode == 0 && P->max_bw <= kBkMaxW)) return batch_band_solve_blk(P, V, R);
    if (mode != 1) return batch_band_solve_win(P, V, R, Lc, Uc);
  }
  constexpr int RG = 8;
  constexpr int D = 8;
  const int ngroups = (R + RG - 1) / RG;
  const int threads = std::max(32, (P->max_bw + 31) / 32 * 32);
  const size_t smem = (size_t)P->max_nodes * RG * sizeof(FT);
  if (threads > 1024 || smem > 200 * 1024) {
    set_detail("batched solve: sub-circuit too large for the batched band solve");
    return VTM_EINVAL;
  }
  VTM_CUDA_TRY(cudaFuncSetAttribute(batch_band_solve_kernel<FT, RG, D>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // FP32 work vectors are row-major ([position][column]), FP64 ones column-major
  const int64_t rs = sizeof(FT) == 4 ? R : 1, cs = sizeof(FT) == 4 ? 1 : P->n;
  batch_band_solve_kernel<FT, RG, D><<<P->nparts * ngroups, threads, smem, P->stream>>>(
      P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(), Lc,
      Uc, V, R, rs, cs);
  P->launch_count++;
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

// ||b_c - A x_c||^2 and ||b_c||^2 for every column (r: residuals out, may be
// NULL); with dfb / dfr set instead, the double-float form on the scaled
// columns (dfx = NULL: x = 0), squares of the scaled values.
static vtm_status batch_norms(vtm_plan_s* P, const double* x, const double* b, double* r, int R,
                              std::vector<double>& rr, std::vector<double>& bb,
                              const float2* dfx = nullptr, const float2* dfb = nullptr,
                              float* v1 = nullptr, float* v2 = nullptr) {
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((P->n + 255) / 256, 152 * 2));
  const int gy = (R + 7) / 8;
  // fixed layout for up to 8 column groups: partials | out[128] | counters
  VTM_TRY(dev_alloc(P->d_bres, ((size_t)gx * 8 * 16 + 2 * 64 + 64) * sizeof(double)));
  double* partials = P->d_bres.as<double>();
  double* out = partials + (size_t)gx * 8 * 16;
  unsigned* counters = reinterpret_cast<unsigned*>(out + 2 * 64);
  if (!P->bres_init) {
    VTM_CUDA_TRY(cudaMemsetAsync(counters, 0, 64 * sizeof(double), P->stream));
    P->bres_init = true;
  }
  if (dfb) {
    // one group of up to 64 columns, 16 rows per block and step
    const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((P->n + 15) / 16, 152 * 8));
    VTM_TRY(dev_alloc(P->d_bres2, ((size_t)gr * 128 + 2 * 64 + 8) * sizeof(double)));
    double* part2 = P->d_bres2.as<double>();
    double* out2 = part2 + (size_t)gr * 128;
    unsigned* cnt2 = reinterpret_cast<unsigned*>(out2 + 2 * 64);
    if (!P->bres2_init) {
      VTM_CUDA_TRY(cudaMemsetAsync(cnt2, 0, 8 * sizeof(double), P->stream));
      P->bres2_init = true;
    }
    batch_residual_rows_kernel<4, 4><<<gr, 256, 0, P->stream>>>(
        P->d_rowptr.as<int64_t>(), P->d_colidx.as<int32_t>(), P->d_vals_df.as<float2>(), dfx, dfb,
        P->d_iperm.as<int32_t>(), v1, v2, P->n, R, gr, part2, cnt2, out2);
    out = out2;
  } else
    batch_residual_norms_kernel<<<gx * gy, 256, 0, P->stream>>>(
        P->d_rowptr.as<int64_t>(), P->d_colidx.as<int32_t>(), P->d_vals.as<double>(), x, b, r, P->n, R,
        gx, gy, partials, counters, out);
  P->launch_count++;
  VTM_CUDA_TRY(cudaGetLastError());
  std::vector<double> h(2 * R);
  VTM_CUDA_TRY(cudaMemcpyAsync(h.data(), out, 2 * R * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  VTM_CUDA_TRY(cudaStreamSynchronize(P->stream));
  rr.resize(R);
  bb.resize(R);
  for (int c = 0; c < R; ++c) {
    rr[c] = h[2 * c];
    bb[c] = h[2 * c + 1];
  }
  return VTM_OK;
}

// A's values as double-float pairs, for the double-float residuals: built
// once per set of values when every nonzero lies within 2^-100 .. 2^100 (the
// scaled products then stay inside FP32's range); vals_df_state 1 = built,
// 2 = out of range.
vtm_status ensure_vals_df(vtm_plan_s* P) {
  if (P->vals_df_state != 0) return VTM_OK;
  bool ok = true;
  for (double v : P->h_vals) {
    int e = 0;
    if (!std::isfinite(v)) ok = false;
    else if (v != 0.0) std::frexp(v, &e);
    if (!ok || e < -100 || e > 100) {
      ok = false;
      break;
    }
  }
  P->vals_df_state = ok ? 1 : 2;
  if (ok) {
    VTM_TRY(dev_alloc(P->d_vals_df, (size_t)std::max<int64_t>(P->nnz, 1) * sizeof(float2)));
    batch_split_kernel<<<grid_n(P->nnz), 256, 0, P->stream>>>(P->d_vals.as<double>(), P->d_vals_df.as<float2>(),
                                                                P->nnz);
    P->launch_count++;
    VTM_CUDA_TRY(cudaGetLastError());
  }
  return VTM_OK;
}

vtm_status solve_batched(vtm_plan_s* P, const double* d_b, double* d_x, int R, double tol,
                         vtm_info* info, bool record_hist) {
  cudaStream_t s = P->stream;
  const int64_t n = P->n;
  const int64_t npt = (int64_t)P->port_node.size();
  const int prec = P->opts.precision;
  if (R > 64) {
    set_detail("batched solve: at most 64 right-hand sides per call");
    return VTM_EINVAL;
  }
  // work items: (tile, block of 64 outputs)
  if (P->item_tile.empty()) {
    for (int32_t t = 0; t < P->nparts; ++t) {
      const int32_t pp = P->port_off[t + 1] - P->port_off[t];
      for (int32_t m = 0; m < pp; m += kMB) {
        P->item_tile.push_back(t);
        P->item_m0.push_back(m);
      }
    }
    VTM_TRY(upload(P->d_item_tile, P->item_tile, s));
    VTM_TRY(upload(P->d_item_m0, P->item_m0, s));
    // longest first: cost of an item ~ p_P * (outputs in the item)
    std::vector<int32_t> order(P->item_tile.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    auto cost = [&](int32_t i) {
      const int32_t t = P->item_tile[i];
      const int64_t pp = P->port_off[t + 1] - P->port_off[t];
      return pp * std::min<int64_t>(kMB, pp - P->item_m0[i]);
    };
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost(a) > cost(b); });
    VTM_TRY(upload(P->d_item_order, order, s));
  }
  const int nitems = (int)P->item_tile.size();
  if (!P->d_iperm.p) VTM_TRY(upload(P->d_iperm, P->iperm, s));
  // tcgen05 work items and the tiled BF16 copy of T_P (BF16 plans; built at
  // the first batched solve after each factorisation)
  if (prec == VTM_PREC_BF16 && P->tc_nitems == 0) {
    std::vector<int32_t> it4;
    std::vector<int64_t> off;
    std::vector<int64_t> cost;
    int64_t o = 0;
    for (int32_t t = 0; t < P->nparts; ++t) {
      const int32_t pp = P->port_off[t + 1] - P->port_off[t];
      if (pp == 0) continue;
      const int nmt = (pp + kTcM - 1) / kTcM, nkc = (pp + kTcK - 1) / kTcK;
      for (int g0 = 0; g0 < nmt; g0 += kTcG) {
        const int ng = std::min(kTcG, nmt - g0);
        it4.insert(it4.end(), {t, g0 * kTcM, ng, nkc});
        off.push_back(o);
        cost.push_back((int64_t)std::min(ng * kTcM, pp - g0 * kTcM) * pp);
        o += (int64_t)ng * nkc * kTcM * kTcK;
      }
    }
    const int nt = (int)off.size();
    std::vector<int32_t> order(nt);
    for (int i = 0; i < nt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    VTM_TRY(upload(P->d_tc_items, it4, s));
    VTM_TRY(upload(P->d_tc_off, off, s));
    VTM_TRY(upload(P->d_tc_order, order, s));
    VTM_TRY(dev_alloc(P->d_Ttc, (size_t)std::max<int64_t>(o, 8) * sizeof(__nv_bfloat16)));
    if (nt > 0)
      pack_tc_kernel<<<nt, 256, 0, s>>>(P->d_T64.as<double>(), P->tabs.T_off.as<int64_t>(),
                                        P->tabs.T_ld.as<int32_t>(), P->tabs.port_off.as<int32_t>(),
                                        P->d_tc_items.as<int4>(), P->d_tc_off.as<int64_t>(),
                                        P->d_Ttc.as<__nv_bfloat16>());
    VTM_CUDA_TRY(cudaGetLastError());
    P->launch_count++;
    P->tc_nitems = nt;
  }
  const bool lowp = prec != VTM_PREC_FP64;
  const size_t wsz = lowp ? sizeof(float) : sizeof(double);
  VTM_TRY(dev_alloc(P->d_bV, (size_t)n * R * sizeof(double)));
  VTM_TRY(dev_alloc(P->d_bstate, 4 * (size_t)std::max<int64_t>(npt, 1) * R * wsz));
  VTM_TRY(dev_alloc(P->d_bc, (size_t)std::max<int64_t>(npt, 1) * R * wsz));
  // per-ticket partials, then the group sums; the group counters follow the
  // control block and are cleared with every upload of it
  const int max_items = std::max(std::max(nitems, P->tc_nitems), 1);
  const int ngroups = (max_items + kBGrp - 1) / kBGrp;
  VTM_TRY(dev_alloc(P->d_bpart, (size_t)(max_items + ngroups) * R * sizeof(double)));
  VTM_TRY(dev_alloc(P->d_btol2, 64 * sizeof(double)));
  VTM_TRY(dev_alloc(P->d_bctrl, sizeof(BatchCtrl) + sizeof(unsigned) * (size_t)ngroups));
  auto upload_bctrl = [&](const BatchCtrl& hc, cudaStream_t st) -> vtm_status {
    VTM_CUDA_TRY(cudaMemcpyAsync(P->d_bctrl.p, &hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    VTM_CUDA_TRY(cudaMemsetAsync(P->d_bctrl.as<BatchCtrl>() + 1, 0, sizeof(unsigned) * (size_t)ngroups, st));
    return VTM_OK;
  };
  VTM_TRY(dev_alloc(P->d_xacc, (size_t)n * R * sizeof(double)));
  double* V = P->d_bV.as<double>();
  // low precision: both banded solves of each refinement step in FP32 (their
  // error is removed by the next step like the sweeps' rounding)
  const bool f32_solves = lowp && P->d_Lc32.p;
  if (f32_solves) VTM_TRY(dev_alloc(P->d_bV32, (size_t)n * R * sizeof(float)));
  // ... and the residuals in double-float when A's nonzeros allow it
  if (f32_solves) VTM_TRY(ensure_vals_df(P));
  // (a solve that stalls on the double-float residual's floor goes on with
  // FP64 residuals: dfres changes once, between refinement steps)
  bool dfres = f32_solves && P->vals_df_state == 1;
  if (dfres) {
    // the residual kernel writes the step's two right-hand sides (FP32, band
    // order) itself: V32 for the first band solve, V32b for the recovery
    VTM_TRY(dev_alloc(P->d_bdf, (size_t)n * R * sizeof(float2)));
    VTM_TRY(dev_alloc(P->d_bV32b, (size_t)n * R * sizeof(float)));
    VTM_TRY(dev_alloc(P->d_xdf, (size_t)n * R * sizeof(float2)));
    VTM_TRY(dev_alloc(P->d_bexp, 2 * 64 * sizeof(int)));
  } else {
    VTM_TRY(dev_alloc(P->d_r, (size_t)n * R * sizeof(double)));
  }
  float* V32 = P->d_bV32.as<float>();
  double* xacc = P->d_xacc.as<double>();
  double* r = P->d_r.as<double>();  // set again when a double-float solve switches to FP64
  float2* bdf = P->d_bdf.as<float2>();
  float* V32b = P->d_bV32b.as<float>();
  float2* xdf = P->d_xdf.as<float2>();
  int* d_emax = P->d_bexp.as<int>();
  int* d_f = d_emax + 64;
  // ||b_r||; double-float residuals: column c scaled by sc[c] = 2^-fexp[c],
  // max |b_c| sc[c] in [1, 2)
  std::vector<double> bnorm(R), rnorm(R), rel(R), sc(R, 1.0);
  std::vector<int> fexp(R, 0);
  VTM_CUDA_TRY(cudaMemsetAsync(xacc, 0, (size_t)n * R * sizeof(double), s));
  std::vector<double> rr2, bb2;
  if (dfres) {
    VTM_CUDA_TRY(cudaMemsetAsync(d_emax, 0, 64 * sizeof(int), s));
    batch_colexp_kernel<<<dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 304)), R),
                          256, 0, s>>>(d_b, n, R, d_emax);
    std::vector<int> emax(R);
    VTM_CUDA_TRY(cudaMemcpyAsync(emax.data(), d_emax, R * sizeof(int), cudaMemcpyDeviceToHost, s));
    VTM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int c = 0; c < R; ++c) {
      fexp[c] = emax[c] > 0 && emax[c] < 0x7ff ? emax[c] - 1023 : 0;
      sc[c] = std::ldexp(1.0, -fexp[c]);
    }
    VTM_CUDA_TRY(cudaMemcpyAsync(d_f, fexp.data(), R * sizeof(int), cudaMemcpyHostToDevice, s));
    batch_split_rm_kernel<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(d_b, d_f, bdf, n, R);
    P->launch_count += 2;
    VTM_TRY(batch_norms(P, nullptr, nullptr, nullptr, R, rr2, bb2, nullptr, bdf, V32, V32b));
    for (int c = 0; c < R; ++c) bnorm[c] = std::ldexp(std::sqrt(bb2[c]), fexp[c]);
  } else {
    VTM_TRY(batch_norms(P, xacc, d_b, r, R, rr2, bb2));
    for (int c = 0; c < R; ++c) bnorm[c] = std::sqrt(bb2[c]);
  }
  for (int c = 0; c < R; ++c) rnorm[c] = bnorm[c];
  info->sweeps = 0;
  info->outer_steps = 0;
  info->relres = 0.0;
  info->first_sweep_converged = 0;
  double inner_tol = P->opts.inner_tol;
  if (inner_tol <= 0) inner_tol = default_inner_tol(prec);
  const int max_outer = prec == VTM_PREC_FP64 ? 4 : P->opts.max_outer;
  int sweeps_left = P->opts.max_sweeps;
  vtm_status result = VTM_ENOCONV;
  bool stalled = false;
  // const / inject on column-major FP64 vectors: one block per 32 ports;
  // row-major FP32 vectors: transposing copies per 32 positions, port-wise
  // kernels along the rows
  const int g1 = grid_n(n * R), g2 = (int)std::max<int64_t>(1, (npt + 31) / 32);
  const int gt = (int)std::max<int64_t>(1, (n + 31) / 32), gp = grid_n(std::max<int64_t>(npt, 1) * R);
  for (int outer = 0; outer < max_outer; ++outer) {
    const double* rhs = outer == 0 ? d_b : r;
    float* Vx = V32;  // the FP32 vector the step's correction ends in
    if (f32_solves) {
      // (double-float residuals: V32 already holds r' in the band order)
      if (!dfres) {
        batch_gather_rm_kernel<double><<<gt, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, V32, n, R);
        P->launch_count++;
      }
      VTM_TRY(batch_band_solve<float>(P, V32, R, P->d_Lc32.as<float>(), P->d_Uc32.as<float>()));
    } else {
      batch_gather_kernel<double><<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, V, n, R);
      P->launch_count++;
      VTM_TRY(batch_band_solve<double>(P, V, R, P->d_Lc.as<double>(), P->d_Uc.as<double>()));
    }
    int kc = 0, flag = 1;
    if (npt > 0) {
      if (f32_solves)
        batch_const_rm_kernel<<<gp, 256, 0, s>>>(P->d_port_pos.as<int32_t>(), P->d_bout32.as<float>(), V32,
                                                 P->d_bc.as<float>(), npt, R);
      else if (lowp)
        batch_const_kernel<double, float><<<g2, 256, 0, s>>>(P->d_port_pos.as<int32_t>(),
                                                            P->d_bout.as<double>(), V,
                                                            P->d_bc.as<float>(), npt, R, n);
      else
        batch_const_kernel<double, double><<<g2, 256, 0, s>>>(P->d_port_pos.as<int32_t>(),
                                                             P->d_bout.as<double>(), V,
                                                             P->d_bc.as<double>(), npt, R, n);
      P->launch_count++;
      std::vector<double> t2(64, 1.0);
      for (int c = 0; c < R; ++c) {
        const double target = tol * bnorm[c];
        const double t_abs = (prec == VTM_PREC_FP64 ? target : std::max(target, inner_tol * rnorm[c])) * sc[c];
        t2[c] = std::max(t_abs * t_abs, 1e-300);
      }
      VTM_CUDA_TRY(cudaMemcpyAsync(P->d_btol2.p, t2.data(), 64 * sizeof(double), cudaMemcpyHostToDevice, s));
      // residual history of column 0 in the first inner solve (the kernels
      // record its squared interface residual; relative to ||rhs_0|| below)
      double* bhist = (record_hist && outer == 0 && P->opts.history && P->opts.history_len > 0)
                          ? P->d_hist.as<double>()
                          : nullptr;
      const int bhist_len = bhist ? P->opts.history_len : 0;
      if (bhist) VTM_CUDA_TRY(cudaMemsetAsync(bhist, 0, bhist_len * sizeof(double), s));
      BatchCtrl h{};
      h.k = 1;
      h.k_max = sweeps_left;
      h.stall = lowp ? 64 : 0;
      h.R = R;
      VTM_TRY(upload_bctrl(h, s));
      VTM_CUDA_TRY(cudaMemsetAsync(P->d_bstate.p, 0, 4 * (size_t)npt * R * wsz, s));
      VTM_CUDA_TRY(cudaStreamSynchronize(s));
      if (sweeps_left <= 0) break;
      // one launch of kernel variant kv (0: CUDA cores, 1: tensor cores) on a
      // persistent grid of at most (SMs x resident CTAs) over the work list
      // variant kv: bit 0 = tensor cores, bit 1 = one work item per CTA instead
      // of a persistent grid (SMs x resident CTAs) over the work list
      // (dry = true: only size the grid, before any graph capture)
      auto launch_batch = [&](int kv, bool dry = false) {
        if (kv == 4) {  // tcgen05 (BF16): persistent CTAs over the tcgen05 work list
          const int key = prec * 8 + kv;
          if (P->batch_grid[key] == 0) {
            cudaFuncSetAttribute(batch_sweep_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
            cudaFuncSetAttribute(batch_sweep_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            int sms = 152, smem_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->device);
            // two CTAs of 256 TMEM columns fill an SM's 512, where their shared
            // memory fits (the occupancy query is not used: it reported one)
            const int per_sm = smem_sm >= 2 * ((int)kTcSmem + 2048) ? 2 : 1;
            P->batch_grid[key] = std::max(1, std::min(P->tc_nitems, per_sm * sms));
          }
          if (dry) return;
          batch_sweep_tc_kernel<<<P->batch_grid[key], kTcThreads, kTcSmem, s>>>(
              P->d_Ttc.as<__nv_bfloat16>(), P->d_tc_items.as<int4>(), P->d_tc_off.as<int64_t>(),
              P->d_tc_order.as<int32_t>(), P->tc_nitems, P->tabs.port_off.as<int32_t>(), P->d_twin.as<int32_t>(),
              P->d_kd.as<double2>(), P->d_run.as<uint8_t>(), P->d_bc.as<float>(), P->d_bstate.as<float>(), npt,
              R, P->d_bctrl.as<BatchCtrl>(), P->d_bpart.as<double>(), P->d_btol2.as<double>(), bhist, bhist_len);
          return;
        }
        auto go = [&](auto* kern, int threads, const auto* T, const auto* cc, auto* st) {
          const int key = prec * 8 + kv;
          if (P->batch_grid[key] == 0) {
            int per_sm = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
            int sms = 152;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
            P->batch_grid[key] = (kv & 2) ? nitems
                                          : std::max(1, std::min(nitems, std::max(per_sm, 1) * sms));
          }
          if (dry) return;
          kern<<<P->batch_grid[key], threads, 0, s>>>(
              T, P->tabs.T_off.as<int64_t>(), P->tabs.T_ld.as<int32_t>(), P->tabs.port_off.as<int32_t>(),
              P->d_item_tile.as<int32_t>(), P->d_item_m0.as<int32_t>(), P->d_item_order.as<int32_t>(),
              nitems, P->d_twin.as<int32_t>(), P->d_kd.as<double2>(), P->d_run.as<uint8_t>(), cc, st,
              npt, R, P->d_bctrl.as<BatchCtrl>(), P->d_bpart.as<double>(), P->d_btol2.as<double>(),
              bhist, bhist_len);
        };
        if (prec == VTM_PREC_BF16 && (kv & 1))
          go(batch_sweep_mma_kernel, 128, P->d_T16.as<__nv_bfloat16>(), P->d_bc.as<float>(),
             P->d_bstate.as<float>());
        // the 16-bit and FP32 CUDA-core sweeps: 8 x 4 outputs per thread (thermal
        // grid, 64 columns: FP32 28.2 against 29.7 ms with 4 x 4, FP16 36.0
        // against 38.4, BF16 36.5 against 38.9)
        else if (prec == VTM_PREC_BF16)
          go(batch_sweep_kernel<__nv_bfloat16, float, float, 8>, 128, P->d_T16.as<__nv_bfloat16>(),
             P->d_bc.as<float>(), P->d_bstate.as<float>());
        else if (prec == VTM_PREC_FP16)
          go(batch_sweep_kernel<__half, float, float, 8>, 128, P->d_T16.as<__half>(), P->d_bc.as<float>(),
             P->d_bstate.as<float>());
        else if (prec == VTM_PREC_FP32)
          go(batch_sweep_kernel<float, float, float, 8>, 128, P->d_T32.as<float>(), P->d_bc.as<float>(),
             P->d_bstate.as<float>());
        else
          go(batch_sweep_kernel<double, double, double>, 256, P->d_T64.as<double>(), P->d_bc.as<double>(),
             P->d_bstate.as<double>());
      };
      // autotune the variant once per plan and precision (tensor cores: BF16
      // with R % 8 == 0; the MMA rounds the waves to the operand type, which
      // for FP16 could overflow on unscaled right-hand sides, so FP16 plans
      // keep the CUDA-core sweep)
      int kv = 0;
      if (P->opts.batch_kernel > 0) {
        // the caller's choice: bit 0 tensor cores (BF16 with R % 8 == 0 only),
        // bit 1 one work item per CTA; 4: tcgen05 (BF16 plans, else CUDA cores)
        kv = P->opts.batch_kernel - 1;
        if (kv == 4 && prec != VTM_PREC_BF16) kv = 0;
        if (kv != 4 && (kv & 1) && !(prec == VTM_PREC_BF16 && R % 8 == 0)) kv &= ~1;
      } else {
        if (P->batch_tuned[prec] == 0 || P->batch_tuned_R[prec] != R) {
          float best = 1e30f;
          for (int cand = 0; cand <= 4; ++cand) {
            if (cand == 4 && prec != VTM_PREC_BF16) continue;
            if (cand != 4 && (cand & 1) && !(prec == VTM_PREC_BF16 && R % 8 == 0)) continue;
            BatchCtrl tt = h;
            tt.k_max = 1 << 30;
            tt.stall = 0;
            VTM_TRY(upload_bctrl(tt, s));
            launch_batch(cand);
            VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
            for (int i = 0; i < 3; ++i) launch_batch(cand);
            VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
            VTM_CUDA_TRY(cudaGetLastError());
            VTM_CUDA_TRY(cudaEventSynchronize(P->evs1));
            float ms = 0.f;
            VTM_CUDA_TRY(cudaEventElapsedTime(&ms, P->evs0, P->evs1));
            P->launch_count += 4;
            if (ms < best) {
              best = ms;
              P->batch_tuned[prec] = cand + 1;
            }
          }
          P->batch_tuned_R[prec] = R;
          VTM_TRY(upload_bctrl(h, s));
          VTM_CUDA_TRY(cudaMemsetAsync(P->d_bstate.p, 0, 4 * (size_t)npt * R * wsz, s));
          if (bhist) VTM_CUDA_TRY(cudaMemsetAsync(bhist, 0, bhist_len * sizeof(double), s));
        }
        kv = P->batch_tuned[prec] - 1;
      }
      P->batch_used = kv + 1;
      // batches of check_every launches replayed from a CUDA graph when the
      // plan has its own stream, and quarter batches for the tail up to the
      // sweeps this refinement step took in the previous solve (the launches
      // up to the one that decides that sweep go out before the first poll)
      const int nb = P->opts.check_every;
      const int snb = std::max(1, nb / 4);
      launch_batch(kv, true);
      cudaGraphExec_t gexec = nullptr, gsmall = nullptr;
      if (P->stream && P->opts.graphs != 1) {
        SweepGraph& G = P->batch_graph[prec];
        const uint64_t key = ((uint64_t)kv << 56) ^ ((uint64_t)nb << 32) ^ ((uint64_t)R << 8) ^
                             (uint64_t)(uintptr_t)P->d_bstate.p ^ ((uint64_t)(uintptr_t)bhist << 3) ^
                             ((uint64_t)bhist_len << 40);
        if (!G.exec || G.key != key) {
          G.reset();
          for (int g = 0; g < 2; ++g) {
            cudaGraph_t graph = nullptr;
            VTM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            for (int i = 0; i < (g ? snb : nb); ++i) launch_batch(kv);
            VTM_CUDA_TRY(cudaStreamEndCapture(s, &graph));
            cudaGraphExec_t& ex = g ? G.small : G.exec;
            if (cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) {
              ex = nullptr;
              cudaGetLastError();
            }
            cudaGraphDestroy(graph);
          }
          if (G.exec) G.key = key;
        }
        gexec = G.exec;
        gsmall = G.small;
      }
      const int step = std::min(outer, 7);
      const int hint = P->batch_hint[prec][step];
      int reps = 1, sreps = 0;
      const int need = hint > 0 ? std::min(hint + 1, sweeps_left + 1) : 0;  // launch k decides sweep k - 1
      if (gexec && need > 0) {
        reps = std::min(need / nb, 64);
        sreps = gsmall ? (need - reps * nb + snb - 1) / snb : 0;
        if (!gsmall && reps * nb < need) ++reps;
        if (reps + sreps == 0) reps = 1;
      }
      // without graphs the first round is the hinted count of single launches
      int first = need;
      int launched = 0;
      BatchCtrl hc{};
      while (true) {
        const int m = gexec ? nb : std::min(first > 0 ? first : nb, sweeps_left + 1 - launched);
        first = 0;
        VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
        if (gexec) {
          for (int i = 0; i < reps; ++i) VTM_CUDA_TRY(cudaGraphLaunch(gexec, s));
          for (int i = 0; i < sreps; ++i) VTM_CUDA_TRY(cudaGraphLaunch(gsmall, s));
        } else {
          for (int i = 0; i < m; ++i) launch_batch(kv);
        }
        VTM_CUDA_TRY(cudaGetLastError());
        const int went = gexec ? reps * nb + sreps * snb : m;
        launched += went;
        VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
        VTM_CUDA_TRY(cudaMemcpyAsync(&hc, P->d_bctrl.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
        VTM_CUDA_TRY(cudaStreamSynchronize(s));
        float bms = 0.f;
        VTM_CUDA_TRY(cudaEventElapsedTime(&bms, P->evs0, P->evs1));
        P->sweep_ms += bms;
        P->sweep_launch_count += went;
        P->launch_count += went;
        reps = 1;
        sreps = 0;
        if (hc.flag || launched > sweeps_left) break;
      }
      flag = hc.flag;
      if (flag == 5) {
        set_detail("vtm_solve (batched): a bounded wait of the tcgen05 sweep ran out");
        return VTM_ETIMEOUT;
      }
      kc = (flag == 1 || flag == 4) ? hc.conv_sweep : std::min(hc.k - 1, sweeps_left);
      P->batch_hint[prec][step] = kc;
      if (bhist) {
        std::vector<double> hh(bhist_len);
        VTM_CUDA_TRY(cudaMemcpyAsync(hh.data(), bhist, bhist_len * sizeof(double), cudaMemcpyDeviceToHost, s));
        VTM_CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < bhist_len; ++i)
          P->opts.history[i] = rnorm[0] > 0 ? std::sqrt(hh[i]) / (rnorm[0] * sc[0]) : 0.0;
      }
      if (outer == 0 && flag == 1) info->first_sweep_converged = kc;
      info->sweeps += kc;
      sweeps_left -= kc;
      const int slot = kc & 1;
      P->launch_count += 2;
      if (f32_solves) {
        // the recovery's right-hand side: r' again (V32b from the residual
        // kernel, or gathered) plus the ports' injections
        if (dfres) Vx = V32b;
        else batch_gather_rm_kernel<double><<<gt, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, V32, n, R);
        batch_inject_rm_kernel<<<gp, 256, 0, s>>>(P->d_port_pos.as<int32_t>(), P->d_run.as<uint8_t>(),
                                                  P->d_beta32.as<float>(),
                                                  P->d_bstate.as<float>() + (size_t)slot * npt * 2 * R, Vx, npt, R);
        VTM_TRY(batch_band_solve<float>(P, Vx, R, P->d_Lc32.as<float>(), P->d_Uc32.as<float>()));
      } else {
        batch_gather_kernel<double><<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, V, n, R);
        if (lowp)
          batch_inject_kernel<double, float><<<g2, 256, 0, s>>>(
              P->d_port_pos.as<int32_t>(), P->d_run.as<uint8_t>(), P->d_beta.as<double>(),
              P->d_bstate.as<float>() + (size_t)slot * npt * 2 * R, V, npt, R, n);
        else
          batch_inject_kernel<double, double><<<g2, 256, 0, s>>>(
              P->d_port_pos.as<int32_t>(), P->d_run.as<uint8_t>(), P->d_beta.as<double>(),
              P->d_bstate.as<double>() + (size_t)slot * npt * 2 * R, V, npt, R, n);
        VTM_TRY(batch_band_solve<double>(P, V, R, P->d_Lc.as<double>(), P->d_Uc.as<double>()));
      }
    } else {
      info->sweeps += 1;
      if (outer == 0) info->first_sweep_converged = 1;
    }
    if (dfres)
      batch_scatter_rm_kernel<true><<<gt, 256, 0, s>>>(P->d_iperm.as<int32_t>(), Vx, xacc, xdf, d_f, n, R,
                                                       outer > 0);
    else if (f32_solves)
      batch_scatter_rm_kernel<false><<<gt, 256, 0, s>>>(P->d_iperm.as<int32_t>(), Vx, xacc, nullptr, nullptr, n,
                                                        R, outer > 0);
    else
      batch_scatter_kernel<double><<<g1, 256, 0, s>>>(P->d_iperm.as<int32_t>(), V, xacc, n, R, outer > 0);
    P->launch_count++;
    VTM_CUDA_TRY(cudaGetLastError());
    info->outer_steps = outer + 1;
    bool all_ok = true, bad = false, stall = false;
    double worst = 0.0;
    if (dfres) VTM_TRY(batch_norms(P, nullptr, nullptr, nullptr, R, rr2, bb2, xdf, bdf, V32, V32b));
    else VTM_TRY(batch_norms(P, xacc, d_b, r, R, rr2, bb2));
    for (int c = 0; c < R; ++c) {
      const double rr = rr2[c];
      const double rprev = rnorm[c];
      rnorm[c] = std::ldexp(std::sqrt(rr), fexp[c]);
      // a column that has not met the tolerance must still gain (safeguard)
      if (rnorm[c] > tol * bnorm[c] && refinement_stalled(prec, rprev, rnorm[c], tol * bnorm[c]))
        stall = true;
      rel[c] = bnorm[c] > 0 ? rnorm[c] / bnorm[c] : rnorm[c];
      worst = std::max(worst, rel[c]);
      if (!std::isfinite(rr)) bad = true;
      if (rnorm[c] > tol * bnorm[c]) all_ok = false;
    }
    if (stall && dfres && !all_ok && !bad) {
      // the double-float residual resolves ||r|| only down to about
      // 2^-48 || |A| |x| ||, and corrections formed from it stop there: the
      // iterate's residual is measured in FP64, and unless that one meets the
      // tolerance the next steps take their right-hand sides from FP64
      // residuals (unscaled columns; the stall test restarts from this norm)
      VTM_TRY(dev_alloc(P->d_r, (size_t)n * R * sizeof(double)));
      r = P->d_r.as<double>();
      std::vector<double> rr64, bb64;
      VTM_TRY(batch_norms(P, xacc, d_b, r, R, rr64, bb64));
      all_ok = true;
      worst = 0.0;
      for (int c = 0; c < R; ++c) {
        rnorm[c] = std::sqrt(rr64[c]);
        if (!(rnorm[c] <= tol * bnorm[c])) all_ok = false;
        if (!std::isfinite(rr64[c])) bad = true;
        worst = std::max(worst, bnorm[c] > 0 ? rnorm[c] / bnorm[c] : rnorm[c]);
        fexp[c] = 0;
        sc[c] = 1.0;
      }
      dfres = false;
      stall = false;
    }
    info->relres = worst;
    if (flag == 3 || bad) {
      result = VTM_EDIVERGED;
      break;
    }
    if (all_ok) {
      result = VTM_OK;
      break;
    }
    if (flag == 2 || sweeps_left <= 0) {
      result = VTM_ENOCONV;
      break;
    }
    if (stall) {
      result = VTM_ENOCONV;
      stalled = true;
      break;
    }
  }
  VTM_CUDA_TRY(cudaMemcpyAsync(d_x, xacc, (size_t)n * R * sizeof(double), cudaMemcpyDeviceToDevice, s));
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  if (result == VTM_ENOCONV)
    set_detail(stalled ? std::string("vtm_solve (batched): refinement stalled (a step cut ||r|| by less than ") +
                             std::to_string((int)refinement_min_gain(prec)) + "x)"
                       : std::string("vtm_solve (batched): tolerance not met"));
  if (result == VTM_EDIVERGED) set_detail("vtm_solve (batched): the iteration diverged");
  return result;
}

}  // namespace vtm
