// VTM sweeps, recovery, FP64 residual and the refinement driver.
//
// One sweep (Sec. VI, Eq. 11 and Eq. 14 with unit line delay) in condensed
// form, for every sub-circuit P at once:
//   w_in(s)  = w_out(twin(s)) of the previous sweep      (zero at sweep 1)
//   w_out_P  = T_P w_in_P + c_P,  c_P(s) = 2 W beta_s x0(l(s)),  x0 = K_P^-1 b_P
// where w_in = W u_twin - i_twin is the wave arriving over the virtual line
// and w_out = W u - i the wave sent back (Eq. 5).  The port voltage of a
// sweep is u = (w_in + w_out)/(2W) and the node voltage behind it follows
// from the twin row of Eq. 11, (2g + W) u - 2g x = w_in.
//
// Residual.  The interior rows of every sub-circuit are solved exactly, so
// b - A x^k is non-zero only at nodes with torn branches, where branch e
// between i (in P) and j (in Q) contributes g (x_i + x_j - 2 u_s); written
// with the waves of both ends, g (x_i + x_j - 2 u_s) =
//   ((W - 2g) u_s + (W + 2g) u_t - w_in_s - w_in_t) / 2.
// The sweep kernel of sweep k evaluates this for sweep k-1 (it reads that
// sweep's waves anyway), sums the ports of each node, squares, reduces per
// tile and finally over tiles in a fixed order (deterministic), and raises a
// device flag when ||r|| <= tol ||b||.  The paper gives no stopping rule;
// this is the relative 2-norm residual after every sweep.
//
// Recovery of the node voltages of the converged sweep:
//   x_P = K_P^-1 (b_P + sum_s beta_s w_in(s) e_l(s)).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <utility>

#include "df.cuh"
#include "ptx.h"
#include "vtm_internal.h"

namespace vtm {

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// Residual term of a torn branch seen from port s (twin t), from the
// (w_in, w_out) pairs of both ends in the plan's wave scaling w / d:
//   ((W - 2g) u_s + (W + 2g) u_t - w_in(s) - w_in(t)) / 2,  u = d (w_in + w_out) / (2W)
//   = d/2 [ (S_s + S_t)/2 - (g/W)(S_s - S_t) - w_in(s) - w_in(t) ],  S = w_in + w_out
// with kd = (g/W, d) of the line.
template <class AT, class KD>
__device__ __forceinline__ AT port_residual(AT wi_s, AT wo_s, AT wi_t, AT wo_t, const KD& kd) {
  const AT Ss = wi_s + wo_s, St = wi_t + wo_t;
  return (AT)0.5 * (AT)kd.y * ((AT)0.5 * (Ss + St) - (AT)kd.x * (Ss - St) - wi_s - wi_t);
}

// Range of the squared residuals in FP32: each tile scales its node
// residuals by 2^-e (e the exponent of the largest) before squaring and the
// FP64 partial is scaled back by 2^2e, so that residuals from 1e-30 to 1e30
// of the right-hand side neither underflow nor overflow.  Power-of-two
// scalings are exact: in FP32's normal range the partial is the same bits as
// the unscaled sum.
__device__ __forceinline__ int pow2_exponent(float v) {  // v >= 0
  const int eb = (int)((__float_as_uint(v) >> 23) & 0xff);
  return min(max(eb - 127, -126), 126);
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <class AT>
struct KdOf {
  using type = float2;
};
template <>
struct KdOf<double> {
  using type = double2;
};

__global__ void gather_perm_kernel(const int32_t* __restrict__ perm, const double* __restrict__ src,
                                   double* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

// dst[perm[i]] (+)= src[i]
template <class VT>
__global__ void scatter_perm_kernel(const int32_t* __restrict__ perm, const VT* __restrict__ src,
                                    double* __restrict__ dst, int64_t n, int accumulate) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (accumulate) dst[perm[i]] += (double)src[i];
    else dst[perm[i]] = (double)src[i];
  }
}

// c(s) = (2 W beta_s / d_s) x0(l(s)) (permuted position pos(s))
template <class WT, class XT>
__global__ void port_const_kernel(const int32_t* __restrict__ port_pos, const double* __restrict__ bout,
                                  const XT* __restrict__ x0, WT* __restrict__ c, int64_t nports) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nports;
       s += (int64_t)gridDim.x * blockDim.x)
    c[s] = (WT)(bout[s] * (double)x0[port_pos[s]]);
}

__global__ void gather_perm_f32_kernel(const int32_t* __restrict__ perm, const double* __restrict__ src,
                                       float* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[perm[i]];
}

// v(l(s)) += sum over the node's ports of beta_s w_in(s); w_in of the chosen
// sweep sits in state[slot][s].x
template <class WT, class VT>
__global__ void inject_kernel(const int32_t* __restrict__ port_pos, const uint8_t* __restrict__ run,
                              const double* __restrict__ beta, const WT* __restrict__ st,
                              VT* __restrict__ v, int64_t nports) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nports;
       s += (int64_t)gridDim.x * blockDim.x) {
    int nr = run[s];
    if (!nr) continue;
    double acc = 0.0;
    for (int q = 0; q < nr; ++q) acc += beta[s + q] * (double)st[2 * (s + q)];
    v[port_pos[s]] = (VT)((double)v[port_pos[s]] + acc);
  }
}

// Fixed-order sum of `count` doubles by one block (result valid in thread 0).
// Loads go out 16 at a time (the sum runs at the end of every sweep, on one
// CTA, so its latency is on the critical path); each thread still adds its
// elements in increasing index order.  With NT > 0 the first NT threads do
// the sum (the order of an NT-thread block); all threads reach the barriers.
template <int NT = 0>
__device__ double block_sum_fixed(const double* __restrict__ a, int64_t count) {
  __shared__ double red[32];
  constexpr int kMLP = 16;
  double acc = 0.0;
  const int nt = NT > 0 ? NT : (int)blockDim.x;
  const int64_t stride = nt;
  for (int64_t base = threadIdx.x; (int)threadIdx.x < nt && base < count; base += kMLP * stride) {
    double v[kMLP];
#pragma unroll
    for (int j = 0; j < kMLP; ++j) {
      const int64_t i = base + j * stride;
      v[j] = i < count ? __ldcg(a + i) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kMLP; ++j) acc += v[j];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = acc;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (nt >> 5); ++i) tot += red[i];
  __syncthreads();
  return tot;
}

// Fixed-order block sum of one float per thread (result valid in thread 0).
__device__ float block_sum_value_f(float v) {
  __shared__ float red3[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red3[w] = v;
  __syncthreads();
  float tot = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red3[i];
  __syncthreads();
  return tot;
}

__device__ double block_sum_value(double v) {
  __shared__ double red2[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red2[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red2[i];
  __syncthreads();
  return tot;
}

// The sweep a CTA of the one-warp-per-tile kernels runs: one counter per CTA
// index after the control block (reset with it), counting the launches this
// CTA index has started.  Every launch has the same grid and each counter is
// touched by one thread per launch, after the wait for the previous launch,
// so it needs no atomic (a shared ticket made every CTA of a sweep queue on
// one address).
__device__ __forceinline__ unsigned take_sweep_number(SweepCtrl* ctrl) {
  unsigned* tk = reinterpret_cast<unsigned*>(ctrl + 1) + blockIdx.x;
  const unsigned t = *reinterpret_cast<volatile unsigned*>(tk) + 1u;
  *tk = t;
  return t;
}

// The last CTA of sweep k closes the sweep: it records the residual of sweep
// k-1 (reduced by that CTA in a fixed order) and decides whether to go on.
// flag 1: converged, 2: sweep limit, 3: diverged or not finite, 4: stalled
// (rounding floor of a low-precision inner solve); a flag already set (a
// bounded wait that timed out) is kept.
__device__ void sweep_decide(SweepCtrl* ctrl, int k, double tot, double* hist, int hist_len) {
  int flag = 0;
  if (k > 1) {
    const int ks = k - 1;
    if (hist && ks <= hist_len) hist[ks - 1] = sqrt(tot / ctrl->bnorm2);
    if (ks == 1) ctrl->first_res2 = tot;
    ctrl->last_res2 = tot;
    if (ks == 1 || tot < 0.81 * ctrl->best_res2) {
      ctrl->best_res2 = tot;
      ctrl->best_k = ks;
    }
    if (!isfinite(tot) || (ks > 1 && tot > 1e12 * ctrl->first_res2 && ctrl->first_res2 > 0)) {
      flag = 3;
    } else if (tot <= ctrl->tol2) {
      flag = 1;
      ctrl->conv_sweep = ks;
    } else if (ctrl->stall > 0 && ks - ctrl->best_k >= ctrl->stall) {
      flag = 4;
      ctrl->conv_sweep = ks;
    }
  }
  if (!flag && k >= ctrl->k_max) flag = 2;
  ctrl->counter = 0u;
  ctrl->k = k + 1;
  __threadfence();
  if (ctrl->flag == 0) ctrl->flag = flag;
}

// The norms of the residual kernels: per-thread sums rr, bb reduced per
// block, then the last block adds the block partials in a fixed order into
// out[0], out[1] and leaves the counter 0.
__device__ void residual_norms_tail(double rr, double bb, double* __restrict__ partials,
                                    unsigned* __restrict__ counter, double* __restrict__ out) {
  double trr = block_sum_value(rr);
  double tbb = block_sum_value(bb);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = trr;
    partials[gridDim.x + blockIdx.x] = tbb;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double a = block_sum_fixed(partials, gridDim.x);
    double c = block_sum_fixed(partials + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      out[0] = a;
      out[1] = c;
      *counter = 0u;
    }
  }
}

// r = b - A x (global order, FP64), ||r||^2 and ||b||^2 reduced in a fixed
// order; out[0] = ||r||^2, out[1] = ||b||^2.  counter must be 0 on entry and
// is left 0.
__global__ void __launch_bounds__(256) residual_kernel(const int64_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b,
                                                       double* __restrict__ r, int64_t n,
                                                       double* __restrict__ partials,
                                                       unsigned* __restrict__ counter,
                                                       double* __restrict__ out) {
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = b[i];
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) acc -= val[q] * x[col[q]];
    if (r) r[i] = acc;
    rr += acc * acc;
    bb += b[i] * b[i];
  }
  residual_norms_tail(rr, bb, partials, counter, out);
}

// The same residual with A in ELL form: entry k of row i at [k n + i]
// (coalesced along the rows), rows shorter than K padded with (0, i).  The
// products are taken in the row's CSR order and a padding entry subtracts an
// exact zero, so r matches the CSR kernel bit for bit (for finite x).  With
// v1 (and v2) r rounded to FP32 also goes to position iperm[i] of those
// vectors: the band-order right-hand sides of an inner solve's two FP32 band
// solves.
template <int K>
__global__ void __launch_bounds__(256) residual_ell_kernel(
    const double* __restrict__ ev, const int32_t* __restrict__ ec, const double* __restrict__ x,
    const double* __restrict__ b, double* __restrict__ r, int64_t n, const int32_t* __restrict__ iperm,
    float* __restrict__ v1, float* __restrict__ v2, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ out) {
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    double av[K];
    int cv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      av[k] = ev[(int64_t)k * n + i];
      cv[k] = ec[(int64_t)k * n + i];
    }
    double acc = bi;
#pragma unroll
    for (int k = 0; k < K; ++k) acc -= av[k] * x[cv[k]];
    if (r) r[i] = acc;
    if (v1) {
      const int pos = iperm[i];
      v1[pos] = (float)acc;
      if (v2) v2[pos] = (float)acc;
    }
    rr += acc * acc;
    bb += bi * bi;
  }
  residual_norms_tail(rr, bb, partials, counter, out);
}

// A in ELL form ([k][n], K entries per row, short rows padded with (0, i))
__global__ void ell_build_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, int64_t n, int K, double* __restrict__ ev,
                                 int32_t* __restrict__ ec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = rowptr[i], len = rowptr[i + 1] - q0;
    for (int k = 0; k < K; ++k) {
      ev[(int64_t)k * n + i] = k < len ? val[q0 + k] : 0.0;
      ec[(int64_t)k * n + i] = k < len ? col[q0 + k] : (int32_t)i;
    }
  }
}
// Host-side launcher of residual_kernel for other translation units; the
// caller provides partials[2*grid], the counter word (0 on entry, left 0)
// and out[2].  Returns the grid it used.
int launch_residual(const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                    const double* b, int64_t n, double* partials, unsigned* counter, double* out,
                    int max_grid, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, max_grid));
  residual_kernel<<<grid, 256, 0, s>>>(rowptr, col, val, x, b, nullptr, n, partials, counter, out);
  return grid;
}

// ---------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------

__device__ __forceinline__ float load_t(const float* p) { return __ldg(p); }
__device__ __forceinline__ double load_t(const double* p) { return __ldg(p); }
__device__ __forceinline__ float load_t(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float load_t(const __half* p) { return __half2float(*p); }

template <class TT, class WT>
__global__ void __launch_bounds__(256) sweep_kernel(
    const TT* __restrict__ T, const int64_t* __restrict__ T_off, const int32_t* __restrict__ T_ld,
    const int32_t* __restrict__ port_off, const int32_t* __restrict__ order,
    const int32_t* __restrict__ twin, const typename KdOf<WT>::type* __restrict__ kd,
    const uint8_t* __restrict__ run, const WT* __restrict__ c, WT* __restrict__ state,
    int64_t nports, SweepCtrl* __restrict__ ctrl, double* __restrict__ partials,
    double* __restrict__ hist, int hist_len, int nparts) {
  using AT = WT;  // accumulation type: FP64 for FP64 waves, FP32 otherwise
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_k, s_flag;
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  const int tile = order[blockIdx.x];
  const int p0 = port_off[tile];
  const int p = port_off[tile + 1] - p0;
  WT* w_in = reinterpret_cast<WT*>(smem_raw);
  AT* rs = reinterpret_cast<AT*>(smem_raw + sizeof(WT) * ((p + 1) & ~1));
  const WT* prev = state + (size_t)((k - 1) & 1) * nports * 2;
  WT* cur = state + (size_t)(k & 1) * nports * 2;
  // gather the incident waves (delay 1) and the residual terms of sweep k-1
  for (int s = threadIdx.x; s < p; s += blockDim.x) {
    const int gs = p0 + s;
    AT wi = 0, rc = 0;
    if (k > 1) {
      const int tw = twin[gs];
      const AT wi_t = (AT)prev[2 * tw], wo_t = (AT)prev[2 * tw + 1];
      const AT wi_s = (AT)prev[2 * gs], wo_s = (AT)prev[2 * gs + 1];
      wi = wo_t;
      rc = port_residual<AT>(wi_s, wo_s, wi_t, wo_t, kd[gs]);
    }
    w_in[s] = (WT)wi;
    rs[s] = rc;
  }
  __syncthreads();
  double sq = 0.0;
  if (k > 1) {
    for (int s = threadIdx.x; s < p; s += blockDim.x) {
      const int nr = run[p0 + s];
      if (nr) {
        double r = 0.0;
        for (int q = 0; q < nr; ++q) r += (double)rs[s + q];
        sq += r * r;
      }
    }
  }
  const double tile_sq = block_sum_value(sq);
  // apply the reflection matrix: w_out(s) = c(s) + sum_t T(s, t) w_in(t)
  const TT* Tb = T + T_off[tile];
  const int ld = T_ld[tile];
  for (int s = threadIdx.x; s < p; s += blockDim.x) {
    AT acc = (AT)c[p0 + s];
    const TT* col = Tb + s;
#pragma unroll 8
    for (int t = 0; t < p; ++t) acc += (AT)load_t(col + (size_t)t * ld) * (AT)w_in[t];
    cur[2 * (p0 + s)] = w_in[s];
    cur[2 * (p0 + s) + 1] = (WT)acc;
  }
  // the last tile to finish reduces the residual of sweep k-1
  if (threadIdx.x == 0) {
    partials[tile] = tile_sq;
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double tot = block_sum_fixed(partials, nparts);
  if (threadIdx.x == 0) sweep_decide(ctrl, k, tot, hist, hist_len);
}

// ---------------------------------------------------------------------------
// the sweep with the reflection matrix staged by the bulk-copy engine
// ---------------------------------------------------------------------------
//
// Same arithmetic as sweep_kernel, persistent over tiles: each CTA handles
// the tiles order[blockIdx.x + m gridDim.x].  Thread 0 streams the T_P^T
// blocks of those tiles, in sequence and across tile boundaries, through a
// ring of kStages shared-memory stages of `ch` rows with cp.async.bulk
// (completion on one mbarrier per stage), so the next tile's matrix is
// already in flight while a tile gathers its incident waves and residual
// terms.  The apply reads T from shared memory with 16-byte vector loads;
// thread (g, l) accumulates VEC consecutive outputs of vector column l over
// the rows t = g (mod G), and the G partial sums are added in a fixed order.

constexpr int kStages = 4;
constexpr uint32_t kWaitPolls = 1u << 24;  // bounded mbarrier wait

template <class TT, int VEC> struct VecLoad;
template <> struct VecLoad<double, 2> {
  __device__ static void load(const double* p, double (&o)[2]) {
    double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};
template <> struct VecLoad<float, 4> {
  __device__ static void load(const float* p, float (&o)[4]) {
    float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <class H> struct VecLoad<H, 8> {  // 16-bit storage (BF16, FP16)
  __device__ static void load(const H* p, float (&o)[8]) {
    uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = Pair16<H>::f2(w[i]);
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

template <class TT, class WT, int VEC, int MAXV>
__global__ void __launch_bounds__(256) sweep_staged_kernel(
    const TT* __restrict__ T, const int64_t* __restrict__ T_off, const int32_t* __restrict__ T_ld,
    const int32_t* __restrict__ port_off, const int32_t* __restrict__ order,
    const int32_t* __restrict__ twin, const typename KdOf<WT>::type* __restrict__ kd,
    const uint8_t* __restrict__ run, const WT* __restrict__ c, WT* __restrict__ state,
    int64_t nports, SweepCtrl* __restrict__ ctrl, double* __restrict__ partials,
    double* __restrict__ hist, int hist_len, int nparts, int ch, int ld_max) {
  using AT = WT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bars[kStages];
  __shared__ int s_k, s_flag, s_timeout;
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
    s_timeout = 0;
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  // shared memory: ring | w_in (ld_max) | rs (ld_max) | red (256 * VEC: one
  // partial per thread and vector element)
  TT* ring = reinterpret_cast<TT*>(smem_raw);
  const size_t stage_elems = (size_t)ch * ld_max;
  WT* w_in = reinterpret_cast<WT*>(smem_raw + kStages * stage_elems * sizeof(TT));
  AT* rs = w_in + ld_max;
  AT* red = rs + ld_max;
  // Producer (thread 0): the chunks of this CTA's tiles (order[blockIdx.x +
  // m gridDim.x], m = 0, 1, ...) in sequence, chunk q into stage q % kStages.
  int pit = blockIdx.x, pc = 0;
  uint32_t issued = 0;
  auto issue_next = [&]() {
    while (pit < nparts) {
      const int tl = order[pit];
      const int pp = port_off[tl + 1] - port_off[tl];
      if (pc * ch < pp) {
        const int ldt = T_ld[tl];
        const int rows = min(ch, pp - pc * ch);
        const uint32_t bytes = (uint32_t)rows * ldt * sizeof(TT);
        uint64_t* bar = &bars[issued % kStages];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(ring + (size_t)(issued % kStages) * stage_elems,
                      T + T_off[tl] + (size_t)pc * ch * ldt, bytes, bar);
        ++pc;
        ++issued;
        return;
      }
      pit += gridDim.x;
      pc = 0;
    }
  };
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < kStages; ++i) issue_next();
  const WT* prev = state + (size_t)((k - 1) & 1) * nports * 2;
  WT* cur = state + (size_t)(k & 1) * nports * 2;
  uint32_t consumed = 0;
  for (int it = blockIdx.x; it < nparts; it += gridDim.x) {
    const int tile = order[it];
    const int p0 = port_off[tile];
    const int p = port_off[tile + 1] - p0;
    const int ld = T_ld[tile];
    // incident waves (delay 1) and residual terms of sweep k-1; the chunks
    // of this tile are already streaming in
    for (int s = tid; s < p; s += blockDim.x) {
      const int gs = p0 + s;
      AT wi = 0, rc = 0;
      if (k > 1) {
        const int tw = twin[gs];
        const AT wi_t = (AT)prev[2 * tw], wo_t = (AT)prev[2 * tw + 1];
        const AT wi_s = (AT)prev[2 * gs], wo_s = (AT)prev[2 * gs + 1];
        wi = wo_t;
        rc = port_residual<AT>(wi_s, wo_s, wi_t, wo_t, kd[gs]);
      }
      w_in[s] = (WT)wi;
      rs[s] = rc;
    }
    __syncthreads();
    AT sq = 0;
    if (k > 1) {
      for (int s = tid; s < p; s += blockDim.x) {
        const int nr = run[p0 + s];
        if (nr) {
          AT r = 0;
          for (int q = 0; q < nr; ++q) r += rs[s + q];
          sq += r * r;
        }
      }
    }
    const double tile_sq = block_sum_value((double)sq);
    if (tid == 0) partials[tile] = tile_sq;
    // apply the reflection matrix from the staged chunks
    const int nv = (p + VEC - 1) / VEC;
    const int L = max(1, min(nv, (int)blockDim.x));
    const int G = blockDim.x / L;
    const int gi = tid / L, li = tid % L;
    AT acc[MAXV][VEC];
#pragma unroll
    for (int m = 0; m < MAXV; ++m)
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[m][e] = 0;
    const int nchunks = (p + ch - 1) / ch;
    for (int ci = 0; ci < nchunks; ++ci, ++consumed) {
      if (tid == 0 &&
          !mbar_wait_bounded(&bars[consumed % kStages], (consumed / kStages) & 1, kWaitPolls))
        s_timeout = 1;
      __syncthreads();
      if (s_timeout) break;
      const TT* st = ring + (size_t)(consumed % kStages) * stage_elems;
      const int r0 = ci * ch, r1 = min(p, r0 + ch);
      if (gi < G) {
        for (int t = r0 + gi; t < r1; t += G) {
          const AT wt = (AT)w_in[t];
          const TT* row = st + (size_t)(t - r0) * ld;
#pragma unroll
          for (int m = 0; m < MAXV; ++m) {
            const int v = li + m * L;
            if (v < nv) {
              AT val[VEC];
              VecLoad<TT, VEC>::load(row + v * VEC, val);
#pragma unroll
              for (int e = 0; e < VEC; ++e) acc[m][e] += val[e] * wt;
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0) issue_next();
    }
    if (s_timeout) break;
    // fixed-order sum over the G row groups (G > 1 only when every thread
    // owns a single vector column, i.e. m = 0)
    if (G > 1) {
      const int cols = L * VEC;
      if (gi < G && li < nv)
#pragma unroll
        for (int e = 0; e < VEC; ++e) red[gi * cols + li * VEC + e] = acc[0][e];
      __syncthreads();
      for (int s = tid; s < p; s += blockDim.x) {
        AT a = (AT)c[p0 + s];
        for (int gg = 0; gg < G; ++gg) a += red[gg * cols + s];
        cur[2 * (p0 + s)] = w_in[s];
        cur[2 * (p0 + s) + 1] = (WT)a;
      }
    } else if (gi == 0) {  // threads past the L vector columns hold no sums
#pragma unroll
      for (int m = 0; m < MAXV; ++m) {
        const int v = li + m * L;
        if (v < nv) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const int s = v * VEC + e;
            if (s < p) {
              cur[2 * (p0 + s)] = w_in[s];
              cur[2 * (p0 + s) + 1] = (WT)(acc[m][e] + (AT)c[p0 + s]);
            }
          }
        }
      }
    }
    __syncthreads();  // w_in, rs and red are reused by the next tile
  }
  if (s_timeout) {
    // wait (bounded) for this CTA's copies still in flight, then report
    if (tid == 0) {
      for (uint32_t q = consumed; q < issued; ++q)
        mbar_wait_bounded(&bars[q % kStages], (q / kStages) & 1, kWaitPolls);
      atomicExch(&ctrl->flag, 5);
    }
    return;
  }
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double tot = block_sum_fixed(partials, nparts);
  if (threadIdx.x == 0) sweep_decide(ctrl, k, tot, hist, hist_len);
}

// ---------------------------------------------------------------------------
// the sweep with 16-byte vector loads straight from HBM
// ---------------------------------------------------------------------------
//
// One CTA per tile; thread (g, l) owns VEC consecutive outputs of vector
// column l and loads its rows t = g (mod G) of T_P^T with 16-byte
// non-allocating loads, all issued before the first FMA of a batch, so each
// thread keeps kBatch loads in flight and the short tiles of a power grid
// need no shared-memory staging.

template <class TT, int VEC> struct VecLoadG;
template <> struct VecLoadG<double, 2> {
  using raw = double2;
  __device__ static raw load(const double* p) { return __ldcs(reinterpret_cast<const double2*>(p)); }
  __device__ static void unpack(const raw& v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }
};
template <> struct VecLoadG<float, 4> {
  using raw = float4;
  __device__ static raw load(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
  __device__ static void unpack(const raw& v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <class H> struct VecLoadG<H, 8> {  // 16-bit storage (BF16, FP16)
  using raw = uint4;
  __device__ static raw load(const H* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
  __device__ static void unpack(const raw& v, float (&o)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = Pair16<H>::f2(w[i]);
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

template <class TT, class WT, int VEC, int NT, int KB>
__global__ void __launch_bounds__(NT) sweep_vec_kernel(
    const TT* __restrict__ T, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const typename KdOf<WT>::type* __restrict__ kd,
    const uint8_t* __restrict__ run, const WT* __restrict__ c, WT* __restrict__ state,
    int64_t nports, SweepCtrl* __restrict__ ctrl, double* __restrict__ partials,
    double* __restrict__ hist, int hist_len, int nparts, int ld_max) {
  using AT = WT;
  using LD = VecLoadG<TT, VEC>;
  constexpr int kBatch = KB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_k, s_flag;
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  // tile descriptor (in launch order) first: the first T loads depend on it only
  const TileDesc dsc = tdesc[blockIdx.x];
  const int tile = dsc.tile;
  const int p0 = dsc.p0;
  const int p = dsc.p;
  const int ld = dsc.ld;
  const TT* Tb = T + dsc.T_off;
  WT* w_in = reinterpret_cast<WT*>(smem_raw);
  AT* rs = w_in + ld_max;
  AT* red = rs + ld_max;
  const int nv = (p + VEC - 1) / VEC;
  const int L = max(1, min(nv, (int)blockDim.x));
  const int G = blockDim.x / L;
  const int gi = tid / L, li = tid % L;
  // first batch of T loads goes out before anything else (it needs no waves)
  typename LD::raw buf[kBatch];
  const bool active = gi < G && li < nv;
#pragma unroll
  for (int b = 0; b < kBatch; ++b) {
    const int t = gi + b * G;
    if (active && t < p) buf[b] = LD::load(Tb + (size_t)t * ld + li * VEC);
  }
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  const WT* prev = state + (size_t)((k - 1) & 1) * nports * 2;
  WT* cur = state + (size_t)(k & 1) * nports * 2;
  for (int s = tid; s < p; s += blockDim.x) {
    const int gs = p0 + s;
    AT wi = 0, rc = 0;
    if (k > 1) {
      const int tw = twin[gs];
      const AT wi_t = (AT)prev[2 * tw], wo_t = (AT)prev[2 * tw + 1];
      const AT wi_s = (AT)prev[2 * gs], wo_s = (AT)prev[2 * gs + 1];
      wi = wo_t;
      rc = port_residual<AT>(wi_s, wo_s, wi_t, wo_t, kd[gs]);
    }
    w_in[s] = (WT)wi;
    rs[s] = rc;
  }
  __syncthreads();
  // node residuals in the wave precision (GB300's FP64 pipe is narrow)
  AT sq = 0;
  if (k > 1) {
    for (int s = tid; s < p; s += blockDim.x) {
      const int nr = run[p0 + s];
      if (nr) {
        AT r = 0;
        for (int q = 0; q < nr; ++q) r += rs[s + q];
        sq += r * r;
      }
    }
  }
  const double tile_sq = block_sum_value((double)sq);
  AT acc[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc[e] = 0;
  if (active) {
    for (int t0 = 0; t0 < p; t0 += kBatch * G) {
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int t = gi + t0 + b * G;
        if (t < p) {
          AT val[VEC];
          LD::unpack(buf[b], val);
          const AT wt = (AT)w_in[t];
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[e] += val[e] * wt;
          const int tn = t + kBatch * G;
          if (tn < p) buf[b] = LD::load(Tb + (size_t)tn * ld + li * VEC);
        }
      }
    }
  }
  if (G > 1) {
    const int cols = L * VEC;
    if (active)
#pragma unroll
      for (int e = 0; e < VEC; ++e) red[gi * cols + li * VEC + e] = acc[e];
    __syncthreads();
    for (int s = tid; s < p; s += blockDim.x) {
      AT a = (AT)c[p0 + s];
      for (int gg = 0; gg < G; ++gg) a += red[gg * cols + s];
      cur[2 * (p0 + s)] = w_in[s];
      cur[2 * (p0 + s) + 1] = (WT)a;
    }
  } else if (active) {
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int s = li * VEC + e;
      if (s < p) {
        cur[2 * (p0 + s)] = w_in[s];
        cur[2 * (p0 + s) + 1] = (WT)(acc[e] + (AT)c[p0 + s]);
      }
    }
  }
  if (tid == 0) {
    partials[tile] = tile_sq;
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double tot = block_sum_fixed(partials, nparts);
  if (threadIdx.x == 0) sweep_decide(ctrl, k, tot, hist, hist_len);
}

// ---------------------------------------------------------------------------
// Packed symmetric sweep.  With scalar W and symmetric A, T_P is symmetric
// (its spectrum is (W - lambda)/(W + lambda), Sec. VIII), so only the 16x16
// blocks on and above the diagonal are stored: about half the bytes of the
// full matrix, which is what an HBM-bound sweep pays for.  A warp takes one
// block (bi, bj) at a time; lane l holds rows l/4 and l/4 + 8, columns
// 4(l%4)..+3, and
//   * adds T_blk w(bj) into the partial of row block bi: a reduce-scatter of
//     its two rows over lane bit 0, then a sum over bit 1;
//   * for bi < bj adds T_blk^T w(bi) into the partial of row block bj: the
//     16-row sums of its four columns are a reduce-scatter over lane bits 4
//     and 3, then a sum over bit 2 (6 shuffles in all, a fixed summation tree).
// part[a][b] holds block b's contribution to row block a; the outputs sum
// them in the fixed order b = 0..nb-1, so every sweep is bitwise repeatable.
// Ways to bring a tile's blocks in: 16-byte register loads a few blocks ahead
// (sweep_sym_kernel), one bulk copy of the whole packed tile into shared
// memory issued before anything else (sweep_symb_kernel), a per-warp ring of
// asynchronous copies (sweep_wsym_kernel).
// ---------------------------------------------------------------------------

// 16-bit storage (BF16, FP16): lane l holds the 16 bytes number l: row l/4,
// columns 4(l%4)..+3, then row l/4 + 8, the same columns (the packing orders
// each 16-bit block that way, so the FP32 block code serves both).
template <class TT>
struct SymLoad {
  using raw = uint4;
  __device__ static raw load(const TT* blk, int lane) {
    return __ldg(reinterpret_cast<const uint4*>(blk) + lane);
  }
  __device__ static raw load_shared(const TT* blk, int lane) {
    return reinterpret_cast<const uint4*>(blk)[lane];
  }
};
// FP32: lane l holds float4 number l (row l/4, columns 4(l%4)..+3) and
// number l + 32 (row l/4 + 8, same columns): each load instruction of the
// warp covers 512 contiguous bytes (no shared-memory bank conflicts).
template <> struct SymLoad<float> {
  struct raw {
    float4 a, b;
  };
  __device__ static raw load(const float* blk, int lane) {
    raw r;
    r.a = __ldg(reinterpret_cast<const float4*>(blk) + lane);
    r.b = __ldg(reinterpret_cast<const float4*>(blk) + lane + 32);
    return r;
  }
  __device__ static raw load_shared(const float* blk, int lane) {
    raw r;
    r.a = reinterpret_cast<const float4*>(blk)[lane];
    r.b = reinterpret_cast<const float4*>(blk)[lane + 32];
    return r;
  }
};

// Per-port inputs that do not depend on the sweep index, loaded at kernel
// start by thread tid for ports tid + j NT (p <= 256): the plan's own tables
// (twin, residual coefficients, node runs), fixed since vtm_factor, and c of
// the current inner solve.
template <int NT>
struct SymPorts {
  static constexpr int PPT = 16 * kSymB / NT;
  int tw[PPT], rn[PPT];
  float2 kq[PPT];
  float cq[PPT];
  __device__ void load_tables(const int32_t* __restrict__ twin, const float2* __restrict__ kd,
                              const uint8_t* __restrict__ run, int p0, int p) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int s = threadIdx.x + j * NT;
      tw[j] = rn[j] = 0;
      kq[j] = make_float2(0.f, 0.f);
      if (s < p) {
        tw[j] = twin[p0 + s];
        kq[j] = kd[p0 + s];
        rn[j] = run[p0 + s];
      }
    }
  }
  __device__ void load_c(const float* __restrict__ c, int p0, int p) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int s = threadIdx.x + j * NT;
      cq[j] = s < p ? c[p0 + s] : 0.f;
    }
  }
  __device__ void load(const int32_t* __restrict__ twin, const float2* __restrict__ kd,
                       const uint8_t* __restrict__ run, const float* __restrict__ c, int p0, int p) {
    load_tables(twin, kd, run, p0, p);
    load_c(c, p0, p);
  }
};

// Programmatic dependent launch (sm_90+): a sweep launched with the
// programmatic-serialization attribute may start while the sweep before it
// finishes.  Before pdl_wait it reads only what no kernel of the solve
// writes (the reflection blocks, the plan's tables); pdl_wait returns once
// the previous grid has completed and its writes are visible.  Without the
// attribute both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Incident waves of the tile (zero past p, the padding of the last block)
// and this thread's share of the squared node residuals of sweep k - 1.
template <int NT>
__device__ __forceinline__ float sym_gather(const SymPorts<NT>& pt, const float* __restrict__ prev,
                                            float* w_in, float* rs, int p0, int p, int nb, int k) {
#pragma unroll
  for (int j = 0; j < SymPorts<NT>::PPT; ++j) {
    const int s = threadIdx.x + j * NT;
    if (s < nb * kSymB) {
      float wi = 0.f, rc = 0.f;
      if (k > 1 && s < p) {
        // L2 reads: in the dataflow kernels other SMs wrote these during this launch
        const float2 wt = __ldcg(reinterpret_cast<const float2*>(prev + 2 * (size_t)pt.tw[j]));
        const float2 ws = __ldcg(reinterpret_cast<const float2*>(prev + 2 * (size_t)(p0 + s)));
        wi = wt.y;
        rc = port_residual<float>(ws.x, ws.y, wt.x, wt.y, pt.kq[j]);
      }
      w_in[s] = wi;
      rs[s] = rc;
    }
  }
  __syncthreads();
  float sq = 0.f;
  if (k > 1) {
#pragma unroll
    for (int j = 0; j < SymPorts<NT>::PPT; ++j) {
      const int s = threadIdx.x + j * NT;
      if (s < p && pt.rn[j]) {
        float rr = 0.f;
        for (int q = 0; q < pt.rn[j]; ++q) rr += rs[s + q];
        sq += rr * rr;
      }
    }
  }
  return sq;
}

// Where a block's partial goes: sink(a, b, i, v) receives element i of block
// b's contribution to row block a.  PartSink stores it for a later fixed-order
// sum over b (several warps per tile); AccSink adds it at once to output a B
// + i (one warp per tile, blocks in row-major order, so each output still
// sums c, then b = 0, 1, ..., nb - 1: the same order as PartSink's sum).
struct PartSink {
  float* part;
  int nb;
  __device__ void operator()(int a, int b, int i, float v) const { part[(a * nb + b) * kSymB + i] = v; }
};
struct AccSink {
  float* acc;
  __device__ void operator()(int a, int, int i, float v) const { acc[a * kSymB + i] += v; }
};

// One 16x16 block (bi, bj) of a warp: the row-block partial T_blk w(bj) and,
// off the diagonal, the column-block partial T_blk^T w(bi) (see above).
template <class Sink>
__device__ __forceinline__ void sym_block(const SymLoad<float>::raw& v, int bi, int bj, int lane,
                                          const float* w_in, const Sink& sink) {
  constexpr int B = kSymB;
  constexpr unsigned FULL = 0xffffffffu;
  const int r1 = lane >> 2, cg = lane & 3;
  // paired FP32 arithmetic (two lanes of a 64-bit register per instruction):
  // each row's four products as two pairs, then the pair's halves added
  const float4 wc = *reinterpret_cast<const float4*>(w_in + bj * B + cg * 4);
  const float2 wc01 = make_float2(wc.x, wc.y), wc23 = make_float2(wc.z, wc.w);
  const float2 pa = __ffma2_rn(make_float2(v.a.z, v.a.w), wc23, __fmul2_rn(make_float2(v.a.x, v.a.y), wc01));
  const float2 pb = __ffma2_rn(make_float2(v.b.z, v.b.w), wc23, __fmul2_rn(make_float2(v.b.x, v.b.y), wc01));
  const float a1 = pa.x + pa.y, a2 = pb.x + pb.y;
  // rows r1 and r1 + 8: sums over the four lanes of a row (bits 0, 1)
  const bool b0 = lane & 1;
  float t = (b0 ? a2 : a1) + __shfl_xor_sync(FULL, b0 ? a1 : a2, 1);
  t += __shfl_xor_sync(FULL, t, 2);
  if (!(lane & 2)) sink(bi, bj, b0 ? r1 + 8 : r1, t);
  if (bi != bj) {
    const float wr1 = w_in[bi * B + r1], wr2 = w_in[bi * B + r1 + 8];
    const float2 w1 = make_float2(wr1, wr1), w2 = make_float2(wr2, wr2);
    const float2 u01 = __ffma2_rn(make_float2(v.b.x, v.b.y), w2, __fmul2_rn(make_float2(v.a.x, v.a.y), w1));
    const float2 u23 = __ffma2_rn(make_float2(v.b.z, v.b.w), w2, __fmul2_rn(make_float2(v.a.z, v.a.w), w1));
    const float u0 = u01.x, u1 = u01.y, u2 = u23.x, u3 = u23.y;
    // columns 4 cg..+3: sums over the eight lanes of a column group (bits 4, 3, 2)
    const bool b4 = lane & 16, b3 = lane & 8;
    float k0 = b4 ? u2 : u0, k1 = b4 ? u3 : u1;
    k0 += __shfl_xor_sync(FULL, b4 ? u0 : u2, 16);
    k1 += __shfl_xor_sync(FULL, b4 ? u1 : u3, 16);
    float t1 = (b3 ? k1 : k0) + __shfl_xor_sync(FULL, b3 ? k0 : k1, 8);
    t1 += __shfl_xor_sync(FULL, t1, 4);
    if (!(lane & 4)) sink(bj, bi, cg * 4 + (b4 ? 2 : 0) + (b3 ? 1 : 0), t1);
  }
}

template <class H, class Sink>
__device__ __forceinline__ void sym_block16(const uint4& raw, int bi, int bj, int lane, const float* w_in,
                                            const Sink& sink) {
  const float2 e0 = Pair16<H>::f2(raw.x), e1 = Pair16<H>::f2(raw.y);
  const float2 e2 = Pair16<H>::f2(raw.z), e3 = Pair16<H>::f2(raw.w);
  SymLoad<float>::raw v;
  v.a = make_float4(e0.x, e0.y, e1.x, e1.y);
  v.b = make_float4(e2.x, e2.y, e3.x, e3.y);
  sym_block(v, bi, bj, lane, w_in, sink);
}

template <class TT, class Sink = PartSink>
__device__ __forceinline__ void sym_apply(const typename SymLoad<TT>::raw& v, int bi, int bj, int lane,
                                          const float* w_in, const Sink& sink) {
  if constexpr (std::is_same<TT, float>::value) sym_block(v, bi, bj, lane, w_in, sink);
  else sym_block16<TT>(v, bi, bj, lane, w_in, sink);
}

// w_out = c + sum of the row block's partials in block order; then the
// tile's residual partial and the last-CTA close of the sweep.
template <int NT>
__device__ __forceinline__ void sym_finish(const SymPorts<NT>& pt, const float* part, const float* w_in,
                                           float* __restrict__ cur, int p0, int p, int nb, int tile,
                                           double tile_sq, int k, SweepCtrl* __restrict__ ctrl,
                                           double* __restrict__ partials, double* __restrict__ hist,
                                           int hist_len, int nparts, bool* s_last) {
  constexpr int B = kSymB;
#pragma unroll
  for (int j = 0; j < SymPorts<NT>::PPT; ++j) {
    const int s = threadIdx.x + j * NT;
    if (s < p) {
      const int a = s / B, rr = s % B;
      float acc = pt.cq[j];
      for (int b = 0; b < nb; ++b) acc += part[(a * nb + b) * B + rr];
      *reinterpret_cast<float2*>(cur + 2 * (size_t)(p0 + s)) = make_float2(w_in[s], acc);
    }
  }
  if (threadIdx.x == 0) {
    partials[tile] = tile_sq;
    __threadfence();
    *s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  const double tot = block_sum_fixed(partials, nparts);
  if (threadIdx.x == 0) sweep_decide(ctrl, k, tot, hist, hist_len);
}

template <class TT, int NT, int KB, int MINB>
__global__ void __launch_bounds__(NT, MINB) sweep_sym_kernel(
    const TT* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state,
    int64_t nports, SweepCtrl* __restrict__ ctrl,
    double* __restrict__ partials, double* __restrict__ hist, int hist_len, int nparts, int pp_max) {
  using LD = SymLoad<TT>;
  constexpr int NW = NT / 32;
  constexpr int B = kSymB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_k, s_flag;
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileDesc dsc = tdesc[blockIdx.x];
  const int tile = dsc.tile, p0 = dsc.p0, p = dsc.p;
  const int nb = (p + B - 1) / B;
  const int nblk = nb * (nb + 1) / 2;
  const TT* Tl = Tp + dsc.Tp_off;
  float* w_in = reinterpret_cast<float*>(smem_raw);
  float* rs = w_in + pp_max;
  float* part = rs + pp_max;
  // the first blocks of T go out before anything else (they need no waves)
  typename LD::raw buf[KB];
#pragma unroll
  for (int b = 0; b < KB; ++b) {
    const int kk = warp + b * NW;
    if (kk < nblk) buf[b] = LD::load(Tl + (size_t)kk * B * B, lane);
  }
  SymPorts<NT> pt;
  pt.load_tables(twin, kd, run, p0, p);
  pdl_launch_dependents();
  pdl_wait();  // the previous sweep's waves, decision and counters
  pt.load_c(c, p0, p);
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  const float* prev = state + (size_t)((k - 1) & 1) * nports * 2;
  float* cur = state + (size_t)(k & 1) * nports * 2;
  const float sq = sym_gather<NT>(pt, prev, w_in, rs, p0, p, nb, k);
  int bi = 0, off = warp;  // block warp + i NW is (bi, bi + off) once off < nb - bi
  for (int base = 0; base < nblk; base += KB * NW) {
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int kk = warp + base + b * NW;
      if (kk < nblk) {
        while (off >= nb - bi) {
          off -= nb - bi;
          ++bi;
        }
        const typename LD::raw v = buf[b];
        const int kn = kk + KB * NW;
        if (kn < nblk) buf[b] = LD::load(Tl + (size_t)kn * B * B, lane);
        sym_apply<TT>(v, bi, bi + off, lane, w_in, PartSink{part, nb});
        off += NW;
      }
    }
  }
  // the residual of sweep k - 1 is reduced after the blocks (its barriers
  // would otherwise hold every warp back before its first block)
  const double tile_sq = (double)block_sum_value_f(sq);
  sym_finish<NT>(pt, part, w_in, cur, p0, p, nb, tile, tile_sq, k, ctrl, partials, hist, hist_len,
                 nparts, &s_last);
}

// The whole packed tile arrives by one bulk copy into shared memory, issued
// first; the wave gather and the residual run while it is in flight.  The
// wait is bounded: on timeout the CTA waits (bounded) for its copy, sets flag
// 5 and leaves the sweep unfinished, which the host reports as VTM_ETIMEOUT.
// The copy is skipped when the flag already reads set; read before pdl_wait
// the flag may still be clear for the one launch after the stop (set flags
// stay set within a batch), and that launch then waits for its copy and
// returns.
template <class TT, int NT>
__global__ void __launch_bounds__(NT) sweep_symb_kernel(
    const TT* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state,
    int64_t nports, SweepCtrl* __restrict__ ctrl,
    double* __restrict__ partials, double* __restrict__ hist, int hist_len, int nparts, int pp_max,
    int tbuf_elems) {
  using LD = SymLoad<TT>;
  constexpr int NW = NT / 32;
  constexpr int B = kSymB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  __shared__ int s_k, s_flag, s_timeout;
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileDesc dsc = tdesc[blockIdx.x];
  const int tile = dsc.tile, p0 = dsc.p0, p = dsc.p;
  const int nb = (p + B - 1) / B;
  const int nblk = nb * (nb + 1) / 2;
  TT* tb = reinterpret_cast<TT*>(smem_raw);
  float* w_in = reinterpret_cast<float*>(smem_raw + (size_t)tbuf_elems * sizeof(TT));
  float* rs = w_in + pp_max;
  float* part = rs + pp_max;
  const uint32_t bytes = (uint32_t)nblk * B * B * sizeof(TT);
  if (tid == 0) {
    // launches past the end of the solve copy nothing
    s_flag = *((volatile int*)&ctrl->flag);
    s_timeout = 0;
    if (!s_flag && bytes) {
      mbar_init(&bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(&bar, bytes);
      bulk_copy_g2s(tb, Tp + dsc.Tp_off, bytes, &bar);
    }
  }
  SymPorts<NT> pt;
  pt.load_tables(twin, kd, run, p0, p);
  pdl_launch_dependents();
  __syncthreads();
  if (s_flag) return;  // no copy was issued
  pdl_wait();  // the previous sweep's waves, decision and counters
  pt.load_c(c, p0, p);
  if (tid == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  __syncthreads();
  if (s_flag) {
    if (tid == 0 && bytes) mbar_wait_bounded(&bar, 0, kWaitPolls);  // the copy lands before the CTA ends
    return;
  }
  const int k = s_k;
  const float* prev = state + (size_t)((k - 1) & 1) * nports * 2;
  float* cur = state + (size_t)(k & 1) * nports * 2;
  const float sq = sym_gather<NT>(pt, prev, w_in, rs, p0, p, nb, k);
  const double tile_sq = (double)block_sum_value_f(sq);
  if (tid == 0 && bytes && !mbar_wait_bounded(&bar, 0, kWaitPolls)) s_timeout = 1;
  __syncthreads();
  if (s_timeout) {
    if (tid == 0) {
      mbar_wait_bounded(&bar, 0, kWaitPolls);
      atomicExch(&ctrl->flag, 5);
    }
    return;
  }
  int bi = 0, off = warp;
  for (int kk = warp; kk < nblk; kk += NW) {
    while (off >= nb - bi) {
      off -= nb - bi;
      ++bi;
    }
    sym_apply<TT>(LD::load_shared(tb + (size_t)kk * B * B, lane), bi, bi + off, lane, w_in,
                  PartSink{part, nb});
    off += NW;
  }
  __syncthreads();
  sym_finish<NT>(pt, part, w_in, cur, p0, p, nb, tile, tile_sq, k, ctrl, partials, hist, hist_len,
                 nparts, &s_last);
}

// ring slots per warp of sweep_wsym_kernel (one block each: 512 B for 16-bit
// entries, 1 KB for FP32; one slot fewer is in flight)
constexpr int kWsymKB16 = 8;
constexpr int kWsymKB32 = 5;
// the dataflow form keeps a tile's state in registers for a whole inner solve:
// 4 warps per CTA and 7 CTAs per SM (up to 72 registers) hold 28 tiles per SM
constexpr int kWflowWarps = 4;
constexpr int kWflowCtasPerSm = 7;

// 16-byte asynchronous copy global -> shared (L2 only), its groups and waits
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// lane's share of one packed block: the bytes it later reads itself (SymLoad)
template <class TT>
__device__ __forceinline__ void copy_block_async(TT* dst, const TT* src, int lane) {
  if constexpr (std::is_same<TT, float>::value) {
    cp_async16(reinterpret_cast<float4*>(dst) + lane, reinterpret_cast<const float4*>(src) + lane);
    cp_async16(reinterpret_cast<float4*>(dst) + lane + 32, reinterpret_cast<const float4*>(src) + lane + 32);
  } else {
    cp_async16(reinterpret_cast<uint4*>(dst) + lane, reinterpret_cast<const uint4*>(src) + lane);
  }
}

// Fixed-order sum of `count` doubles by the 128 threads t = 0..127 of a
// named barrier group (bar id 1): the order of block_sum_fixed<128>, for four
// warps that run beside others.  Valid in t = 0.
__device__ double group128_sum_fixed(const double* __restrict__ a, int64_t count, int t, double* red) {
  constexpr int kMLP = 16;
  double acc = 0.0;
  for (int64_t base = t; base < count; base += kMLP * 128) {
    double v[kMLP];
#pragma unroll
    for (int j = 0; j < kMLP; ++j) {
      const int64_t i = base + j * 128;
      v[j] = i < count ? __ldcg(a + i) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kMLP; ++j) acc += v[j];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((t & 31) == 0) red[t >> 5] = acc;
  asm volatile("bar.sync 1, 128;" ::: "memory");
  double tot = 0.0;
  if (t == 0)
    for (int i = 0; i < 4; ++i) tot += red[i];
  return tot;
}

// One warp per tile: the warp takes all of its tile's packed blocks (in
// column-major order, see the block loop) and adds the partials into the
// tile's outputs itself, with the next KB - 1 blocks of the tile in flight
// into a ring of KB shared-memory slots (each lane copies, and later reads,
// its own bytes of a block, so no warp barrier guards the ring).
// There is no CTA barrier inside a tile; a CTA holds up to 32 tiles, dealt
// round the CTAs (tile warp x gridDim + CTA), so every tile of a
// few-thousand-tile plan is resident at once (one CTA of 27 tile warps per
// SM for 4096 tiles on 152 SMs) and each SM carries the same mix of tile
// sizes: a sweep streams the blocks without waves of CTAs, each tile's chain
// of dependent loads overlapped by all the others.
// The launch decides nothing about its own sweep: the four service warps
// after the tile warps of CTA 0 sum the residual partials of the previous
// sweep and take its decision while the tiles run, so no last-CTA tail sits
// on the critical path of a sweep.  The stop therefore lands one launch
// later, and the waves live in three slots (sweep k writes slot k mod 3),
// so the iterate a decision names survives the sweep after it.  Each launch
// takes its sweep number from a ticket (CTAs of launches past a stop leave
// before taking one).
// The products are those of the other packed kernels; the column partials
// are summed over a block column before their cross-lane reduction, so the
// rounding of the outputs differs from theirs (the order is fixed: every run
// is bitwise repeatable).  Each tile's squared residual is reduced as four
// 32-thread groups (virtual thread lane + 32 v owns ports lane + 32 v + 128 j)
// and the tiles' partials in the order of a 128-thread block, as in kernel 5.
// PPL ports per lane: 4 (tiles of at most 128 ports) or 8 (256).
template <class TT, int KB, int PPL>
__global__ void __launch_bounds__(1024, 1) sweep_wsym_kernel(
    const TT* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state3,
    int64_t nports, SweepCtrl* __restrict__ ctrl,
    double* __restrict__ partials2, double* __restrict__ hist, int hist_len, int nparts, int pp_max) {
  using LD = SymLoad<TT>;
  constexpr int B = kSymB;
  static_assert(PPL == 4 || PPL == 8, "ports per lane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_k, s_flag;
  __shared__ double s_red[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (int)(blockDim.x >> 5) - 4;  // tile warps; the last four serve
  // launches past the end of the solve copy nothing (a set flag stays set
  // within a batch; read before pdl_wait a clear one may be stale)
  if (tid == 0) s_flag = *((volatile int*)&ctrl->flag);
  __syncthreads();
  if (s_flag) return;
  const bool tile_warp = warp < nw;
  const int g = warp * gridDim.x + blockIdx.x;  // tiles dealt round the CTAs
  const bool valid = tile_warp && g < nparts;
  TileDesc dsc{};
  if (valid) dsc = tdesc[g];
  const int p0 = dsc.p0, p = valid ? dsc.p : 0;
  const int nb = (p + B - 1) / B;
  const int nblk = nb * (nb + 1) / 2;
  const TT* Tl = Tp + dsc.Tp_off;
  TT* ring = reinterpret_cast<TT*>(smem_raw +
                                   (size_t)(tile_warp ? warp : 0) * (KB * B * B * sizeof(TT) + 12 * (size_t)pp_max));
  float* w_in = reinterpret_cast<float*>(ring + KB * B * B);
  float* rs = w_in + pp_max;
  float* acc = rs + pp_max;
  // the ring's first blocks and the plan's port tables go out before the wait
  int tw[PPL];
  uint32_t rn4[PPL / 4];  // node-run lengths, one byte per port
  // the copy stream follows the column-major block order: block (pbi, pbj)
  // is number pidx of the row-major packed tile; pq counts copies issued
  int pbi = 0, pbj = 0, pidx = 0, pq = 0;
  auto issue_next = [&]() {
    if (pq < nblk) {
      copy_block_async(ring + (pq % KB) * B * B, Tl + (size_t)pidx * B * B, lane);
      if (pbi < pbj) {
        pidx += nb - 1 - pbi;
        ++pbi;
      } else {
        ++pbj;
        pbi = 0;
        pidx = pbj;
      }
    }
    ++pq;
    cp_async_commit_group();
  };
  if (tile_warp) {
#pragma unroll
    for (int b = 0; b < KB - 1; ++b) issue_next();
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      tw[m] = s < p ? twin[p0 + s] : 0;
    }
#pragma unroll
    for (int j = 0; j < PPL / 4; ++j) {
      uint32_t r = 0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int s = lane + 32 * (v + 4 * j);
        if (s < p) r |= (uint32_t)run[p0 + s] << (8 * v);
      }
      rn4[j] = r;
    }
  }
  pdl_launch_dependents();
  pdl_wait();  // the previous sweep's waves, partials and decision
  if (tid == 0) {
    s_flag = *((volatile int*)&ctrl->flag);
    if (!s_flag) s_k = (int)take_sweep_number(ctrl);
  }
  __syncthreads();
  if (s_flag) {
    cp_async_wait_group<0>();  // no copy into shared memory outlives the CTA
    return;
  }
  const int k = s_k;
  if (!tile_warp) {  // service warps: CTA 0 decides on the previous sweep
    if (blockIdx.x != 0 || k < 2) return;
    const int t = tid - nw * 32;
    const double tot = group128_sum_fixed(partials2 + (size_t)((k - 1) & 1) * nparts, nparts, t, s_red);
    if (t == 0) sweep_decide(ctrl, k - 1, tot, hist, hist_len);
    return;
  }
  const float* prev = state3 + (size_t)((k - 1) % 3) * nports * 2;
  float* cur = state3 + (size_t)(k % 3) * nports * 2;
  // incident waves and residual terms of sweep k - 1; the outputs start at c
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    if (s < nb * B) {
      float wi = 0.f, rc = 0.f, c0 = 0.f;
      if (s < p) {
        c0 = c[p0 + s];
        if (k > 1) {
          const float2 wt = *reinterpret_cast<const float2*>(prev + 2 * (size_t)tw[m]);
          const float2 ws = *reinterpret_cast<const float2*>(prev + 2 * (size_t)(p0 + s));
          wi = wt.y;
          rc = port_residual<float>(ws.x, ws.y, wt.x, wt.y, kd[p0 + s]);
        }
      }
      w_in[s] = wi;
      rs[s] = rc;
      acc[s] = c0;
    }
  }
  __syncwarp();
  float tile_sq = 0.f;  // lane 0: the four groups in order, scaled by 2^-2 tile_e
  int tile_e = 0;
  if (k > 1) {
    float rrv[PPL];
    float rmax = 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int j = 0; j < PPL / 4; ++j) {
        const int s = lane + 32 * (v + 4 * j);
        const int nr = (rn4[j] >> (8 * v)) & 0xff;
        float rr = 0.f;
        if (s < p && nr)
          for (int q = 0; q < nr; ++q) rr += rs[s + q];
        rrv[v * (PPL / 4) + j] = rr;
        rmax = fmaxf(rmax, fabsf(rr));
      }
    tile_e = pow2_exponent(warp_max(rmax));
    const float rsc = pow2f(-tile_e);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float sq = 0.f;
#pragma unroll
      for (int j = 0; j < PPL / 4; ++j) {
        const int s = lane + 32 * (v + 4 * j);
        const int nr = (rn4[j] >> (8 * v)) & 0xff;
        if (s < p && nr) {
          const float rr = rrv[v * (PPL / 4) + j] * rsc;
          sq += rr * rr;
        }
      }
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
      tile_sq += sq;
    }
  }
  // Blocks in column-major order over the upper triangle: column bj takes
  // (0, bj), (1, bj), ..., (bj, bj).  Each block's row partial T_blk w(bj)
  // is reduced at once into its row block bi; its column partial T_blk^T
  // w(bi) only accumulates in registers (ca01, ca23: this lane's two rows'
  // products for its four columns, summed over bi), reduced across the eight
  // lanes of a column group once per column, after the diagonal block.  Row
  // outputs have fixed owner lanes (bit 1 clear), column outputs too (bit 2
  // clear), so two warp barriers per column order every cross-lane update.
  const int r1 = lane >> 2, cg = lane & 3;
  const bool b0 = lane & 1, b4 = lane & 16, b3 = lane & 8;
  const bool row_owner = !(lane & 2), col_owner = !(lane & 4);
  const int myrow = b0 ? r1 + 8 : r1;
  const int mycol = cg * 4 + (b4 ? 2 : 0) + (b3 ? 1 : 0);
  constexpr unsigned FULL = 0xffffffffu;
  float2 ca01 = make_float2(0.f, 0.f), ca23 = make_float2(0.f, 0.f);
  int bi = 0, bj = 0;
  for (int kk = 0; kk < nblk; ++kk) {
    issue_next();
    cp_async_wait_group<KB - 1>();  // this lane's bytes of block kk have landed
    SymLoad<float>::raw v;
    if constexpr (std::is_same<TT, float>::value) {
      v = LD::load_shared(ring + (kk % KB) * B * B, lane);
    } else {
      const uint4 raw = LD::load_shared(ring + (kk % KB) * B * B, lane);
      const float2 e0 = Pair16<TT>::f2(raw.x), e1 = Pair16<TT>::f2(raw.y);
      const float2 e2 = Pair16<TT>::f2(raw.z), e3 = Pair16<TT>::f2(raw.w);
      v.a = make_float4(e0.x, e0.y, e1.x, e1.y);
      v.b = make_float4(e2.x, e2.y, e3.x, e3.y);
    }
    const float2 a01 = make_float2(v.a.x, v.a.y), a23 = make_float2(v.a.z, v.a.w);
    const float2 b01 = make_float2(v.b.x, v.b.y), b23 = make_float2(v.b.z, v.b.w);
    {  // row partial of rows r1, r1 + 8: pairs, then a sum over the row's four lanes
      const float4 wc = *reinterpret_cast<const float4*>(w_in + bj * B + cg * 4);
      const float2 wc01 = make_float2(wc.x, wc.y), wc23 = make_float2(wc.z, wc.w);
      const float2 pa = __ffma2_rn(a23, wc23, __fmul2_rn(a01, wc01));
      const float2 pb = __ffma2_rn(b23, wc23, __fmul2_rn(b01, wc01));
      const float x1 = pa.x + pa.y, x2 = pb.x + pb.y;
      float t = (b0 ? x2 : x1) + __shfl_xor_sync(FULL, b0 ? x1 : x2, 1);
      t += __shfl_xor_sync(FULL, t, 2);
      if (row_owner) acc[bi * B + myrow] += t;
    }
    if (bi != bj) {
      const float wr1 = w_in[bi * B + r1], wr2 = w_in[bi * B + r1 + 8];
      const float2 w1 = make_float2(wr1, wr1), w2 = make_float2(wr2, wr2);
      ca01 = __ffma2_rn(b01, w2, __ffma2_rn(a01, w1, ca01));
      ca23 = __ffma2_rn(b23, w2, __ffma2_rn(a23, w1, ca23));
      ++bi;
    } else {
      __syncwarp();  // the diagonal block's row partial is in before the column's
      if (bj > 0) {
        // columns 4 cg..+3: sums over the eight lanes of a column group (bits 4, 3, 2)
        float k0 = b4 ? ca23.x : ca01.x, k1 = b4 ? ca23.y : ca01.y;
        k0 += __shfl_xor_sync(FULL, b4 ? ca01.x : ca23.x, 16);
        k1 += __shfl_xor_sync(FULL, b4 ? ca01.y : ca23.y, 16);
        float t1 = (b3 ? k1 : k0) + __shfl_xor_sync(FULL, b3 ? k0 : k1, 8);
        t1 += __shfl_xor_sync(FULL, t1, 4);
        if (col_owner) acc[bj * B + mycol] += t1;
      }
      __syncwarp();  // and the column partial before later rows add to this block
      ca01 = ca23 = make_float2(0.f, 0.f);
      ++bj;
      bi = 0;
    }
  }
  cp_async_wait_group<0>();
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    if (s < p) *reinterpret_cast<float2*>(cur + 2 * (size_t)(p0 + s)) = make_float2(w_in[s], acc[s]);
  }
  if (valid && lane == 0) partials2[(size_t)(k & 1) * nparts + dsc.tile] = (double)tile_sq * pow2d(2 * tile_e);
}

// ---------------------------------------------------------------------------
// Packed symmetric sweep with the block products on the tensor cores (kernel
// 11; 16-bit blocks, tiles of at most 128 ports).  Kernel 9's organisation
// (one warp per tile, one CTA per SM with four service warps, three wave
// slots, the decision on sweep k - 1 taken by CTA 0's service warps), with
// each 16x16 block applied by warp MMAs (mma.sync m16n8k16, FP32 accumulate):
// the row part T_blk w(bj) and the column part T_blk^T w(bi) of block (bi, bj)
// are one MMA each.  Their B operand carries the tile's incident waves, scaled
// by a power of two sc (largest |sc w| in [2^13, 2^14)), as two 16-bit numbers
// hi = rn(sc w) in column 0 and lo = rn(sc w - hi) in column 1 (zero
// elsewhere): column 0 + column 1 of the product is T_blk (sc w) with the
// waves kept to 22 (FP16) or 16 (BF16) bits, against the 11 / 8 bits of T_P's
// own storage.  Lane l, g = l / 4, t = l % 4:
//   * stored block (the 16-bit layout of the other packed kernels): words
//     x = T[g][4t, 4t+1], y = T[g][4t+2, 4t+3], z = T[g+8][4t, 4t+1],
//     w = T[g+8][4t+2, 4t+3];
//   * row part: A = {x, z, y, w}, so MMA index k = 2t+e stands for block
//     column 4t+e and k = 8+2t+e for 4t+2+e; B (lanes 0-3 hi, 4-7 lo) holds
//     (w[4t], w[4t+1]) and (w[4t+2], w[4t+3]); output row r is block row r;
//   * column part: A = the 8x8 transposes (movmatrix) of x, y, z, w, so k is
//     the block row and MMA row m stands for block column kx(m) = 4(m/2) +
//     m%2 (m < 8) or ky(m-8) = 4((m-8)/2) + 2 + m%2 (m >= 8); B holds
//     (w[2t], w[2t+1]) and (w[8+2t], w[9+2t]).
// The output of both sits in lanes 4q: rows q and q + 8, (hi, lo) pairs.
// Blocks run column by column as in kernel 9: the column part of every block
// of column bj, and the diagonal block (symmetric, so through the same
// transposed form), accumulate in one MMA accumulator, stored once per
// column; each row part is added at once to its row block's (hi, lo) pair in
// shared memory by the lanes that own those rows.
// ---------------------------------------------------------------------------

template <class TT>
struct Mma16;
template <>
struct Mma16<__half> {
  __device__ static void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                             uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  // (hi, lo) of a pair of scaled waves, as two packed 16-bit pairs
  __device__ static uint2 split(float v0, float v1) {
    const __half2 h = __floats2half2_rn(v0, v1);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(v0 - f.x, v1 - f.y);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&h), *reinterpret_cast<const uint32_t*>(&l));
  }
};
template <>
struct Mma16<__nv_bfloat16> {
  __device__ static void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                             uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  __device__ static uint2 split(float v0, float v1) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 f = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - f.x, v1 - f.y);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&h), *reinterpret_cast<const uint32_t*>(&l));
  }
};
// transpose of an 8x8 16-bit matrix held one row-pair word per lane
__device__ __forceinline__ uint32_t movm_trans(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}

// f(integral_constant<int, I>) for I = 0 .. N - 1, unrolled at compile time
template <int N, int I = 0, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<N, I + 1>(f);
  }
}

constexpr int kWmmaNB = 8;  // block rows of the largest tile (128 ports)
constexpr int kWmmaPD = 4;  // blocks loaded ahead per lane

template <class TT, int PD>
__global__ void __launch_bounds__(1024, 1) sweep_wmma_kernel(
    const TT* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state3,
    int64_t nports, SweepCtrl* __restrict__ ctrl,
    double* __restrict__ partials2, double* __restrict__ hist, int hist_len, int nparts, int pp_max) {
  using M = Mma16<TT>;
  constexpr int B = kSymB;
  constexpr int PPL = 4;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_k, s_flag;
  __shared__ double s_red[4];
  __shared__ uint2 s_zero[kWmmaNB * 8];  // the B operand rows of lanes 8-31
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (int)(blockDim.x >> 5) - 4;  // tile warps; the last four serve
  if (tid == 0) s_flag = *((volatile int*)&ctrl->flag);
  if (tid < kWmmaNB * 8) s_zero[tid] = make_uint2(0u, 0u);
  __syncthreads();
  if (s_flag) return;
  const bool tile_warp = warp < nw;
  const int g = warp * gridDim.x + blockIdx.x;  // tiles dealt round the CTAs
  const bool valid = tile_warp && g < nparts;
  TileDesc dsc{};
  if (valid) dsc = tdesc[g];
  const int p0 = dsc.p0, p = valid ? dsc.p : 0;
  const int nb = (p + B - 1) / B;
  const TT* Tl = Tp + dsc.Tp_off;
  // per warp: w_in, residual terms, c, the (hi, lo) row sums and the B
  // operands of the column and row parts (lanes 0-7, a row of eight per
  // block row)
  unsigned char* wbase = smem_raw + (size_t)(tile_warp ? warp : 0) * (20 * (size_t)pp_max + 128 * kWmmaNB);
  float* w_in = reinterpret_cast<float*>(wbase);
  float* rs = w_in + pp_max;
  float* cs = rs + pp_max;
  float2* acc2 = reinterpret_cast<float2*>(cs + pp_max);
  uint2* bcs = reinterpret_cast<uint2*>(acc2 + pp_max);
  uint2* brs = bcs + 8 * kWmmaNB;
  // this lane's 16 bytes of block q (column-major block order: column bj
  // holds blocks (0, bj) .. (bj, bj)) of the row-major packed tile, while it
  // exists (bj < nb), loaded PD blocks ahead into register slot q mod PD.
  // Plain loads rather than asynchronous copies into shared memory: for a
  // tile set that stays in L2 between sweeps they deliver about 1.5 times
  // the bandwidth.  The loads are ordered instructions, so the prefetch
  // distance is what the code says.
  uint4 pf[PD];
  auto issue = [&](auto qc) {
    constexpr int q = decltype(qc)::value;
    constexpr int bj = q < 1 ? 0 : q < 3 ? 1 : q < 6 ? 2 : q < 10 ? 3 : q < 15 ? 4 : q < 21 ? 5 : q < 28 ? 6 : q < 36 ? 7 : 8;
    constexpr int bi = q - bj * (bj + 1) / 2;
    if (bj < nb) {
      const int pidx = bi * nb - bi * (bi - 1) / 2 + bj - bi;
      const uint4* src = reinterpret_cast<const uint4*>(Tl + (size_t)pidx * B * B) + lane;
      uint4& d = pf[q % PD];
      asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                   : "=r"(d.x), "=r"(d.y), "=r"(d.z), "=r"(d.w)
                   : "l"(src));
    }
  };
  int tw[PPL];
  uint32_t rn4 = 0;  // node-run lengths, one byte per port
  if (tile_warp) {
    static_for<PD>([&](auto qc) { issue(qc); });
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      tw[m] = s < p ? twin[p0 + s] : 0;
      if (s < p) rn4 |= (uint32_t)run[p0 + s] << (8 * m);
    }
  }
  pdl_launch_dependents();
  pdl_wait();  // the previous sweep's waves, partials and decision
  if (tid == 0) {
    s_flag = *((volatile int*)&ctrl->flag);
    if (!s_flag) s_k = (int)take_sweep_number(ctrl);
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  if (!tile_warp) {  // service warps: CTA 0 decides on the previous sweep
    if (blockIdx.x != 0 || k < 2) return;
    const int t = tid - nw * 32;
    const double tot = group128_sum_fixed(partials2 + (size_t)((k - 1) & 1) * nparts, nparts, t, s_red);
    if (t == 0) sweep_decide(ctrl, k - 1, tot, hist, hist_len);
    return;
  }
  const float* prev = state3 + (size_t)((k - 1) % 3) * nports * 2;
  float* cur = state3 + (size_t)(k % 3) * nports * 2;
  // incident waves and residual terms of sweep k - 1, c, and the waves'
  // scale.  Every port's loads go out before any shared-memory store, so the
  // lane waits for one round trip, not one per port.
  float c0v[PPL];
  float2 wtv[PPL], wsv[PPL], kqv[PPL];
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    c0v[m] = 0.f;
    wtv[m] = wsv[m] = kqv[m] = make_float2(0.f, 0.f);
    if (s < p) {
      c0v[m] = c[p0 + s];
      if (k > 1) {
        wtv[m] = *reinterpret_cast<const float2*>(prev + 2 * (size_t)tw[m]);
        wsv[m] = *reinterpret_cast<const float2*>(prev + 2 * (size_t)(p0 + s));
        kqv[m] = kd[p0 + s];
      }
    }
  }
  float amax = 0.f;
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    if (s < nb * B) {
      float wi = 0.f, rc = 0.f;
      if (s < p && k > 1) {
        wi = wtv[m].y;
        rc = port_residual<float>(wsv[m].x, wsv[m].y, wtv[m].x, wtv[m].y, kqv[m]);
      }
      w_in[s] = wi;
      rs[s] = rc;
      cs[s] = c0v[m];
      amax = fmaxf(amax, fabsf(wi));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
  // sc = 2^(13 - E) for |w| max = 1.f x 2^E (biased exponent clamped so that
  // sc and 1 / sc are both normal: their product is exactly one)
  const int se = min(max(267 - (int)((__float_as_uint(amax) >> 23) & 0xff), 1), 253);
  const float sc = __uint_as_float((uint32_t)se << 23), isc = __uint_as_float((uint32_t)(254 - se) << 23);
  __syncwarp();
  float tile_sq = 0.f;  // lane 0: the four groups in order, scaled by 2^-2 tile_e
  int tile_e = 0;
  if (k > 1) {
    float rrv[PPL];
    float rmax = 0.f;
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      const int nr = (rn4 >> (8 * m)) & 0xff;
      float rr = 0.f;
      if (s < p && nr)
        for (int q = 0; q < nr; ++q) rr += rs[s + q];
      rrv[m] = rr;
      rmax = fmaxf(rmax, fabsf(rr));
    }
    tile_e = pow2_exponent(warp_max(rmax));
    const float rsc = pow2f(-tile_e);
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      float sq = 0.f;
      const int s = lane + 32 * m;
      const int nr = (rn4 >> (8 * m)) & 0xff;
      if (s < p && nr) {
        const float rr = rrv[m] * rsc;
        sq = rr * rr;
      }
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(FULL, sq, o);
      tile_sq += sq;
    }
  }
  // B operands, one row of eight per block row r: entry 8 r + f for lane f
  // < 8 (f < 4: hi, f >= 4: lo, t = f % 4); the column parts take (w[2t],
  // w[2t+1]) and (w[8+2t], w[9+2t]) of block row r, the row parts (w[4t],
  // w[4t+1]) and (w[4t+2], w[4t+3]).  Two entries per lane; lanes 0-7 read
  // back their own column, the others read zeros.
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = lane + 32 * h, r = e >> 3, f = e & 7, ft = f & 3;
    if (r < nb) {
      const float* wr = w_in + r * B;
      const float2 u = *reinterpret_cast<const float2*>(wr + 2 * ft);
      const float2 v = *reinterpret_cast<const float2*>(wr + 8 + 2 * ft);
      const float4 q = *reinterpret_cast<const float4*>(wr + 4 * ft);
      const uint2 su = M::split(u.x * sc, u.y * sc), sv = M::split(v.x * sc, v.y * sc);
      const uint2 s01 = M::split(q.x * sc, q.y * sc), s23 = M::split(q.z * sc, q.w * sc);
      bcs[e] = f >= 4 ? make_uint2(su.y, sv.y) : make_uint2(su.x, sv.x);
      brs[e] = f >= 4 ? make_uint2(s01.y, s23.y) : make_uint2(s01.x, s23.x);
    }
  }
  __syncwarp();
  const int gq = lane >> 2, t4 = lane & 3;
  const bool bl = gq < 2;
  const uint2* bsrc = bl ? bcs + lane : s_zero;
  const uint2* rsrc = bl ? brs + lane : s_zero;
  const bool owner = t4 == 0;  // lanes 4q: rows q and q + 8 of each output
  const int kxq = 4 * (gq >> 1) + (gq & 1), kyq = kxq + 2;
  static_for<kWmmaNB>([&](auto jc) {
    constexpr int bj = decltype(jc)::value;
    if (bj < nb) {
      const uint2 br = rsrc[bj * 8];  // B operand of the row parts: w(bj)
      float dc[4] = {0.f, 0.f, 0.f, 0.f};
      static_for<bj + 1>([&](auto ic) {
        constexpr int bi = decltype(ic)::value;
        constexpr int kk = bj * (bj + 1) / 2 + bi;
        const uint4 raw = pf[kk % PD];
        issue(std::integral_constant<int, kk + PD>{});
        if constexpr (bi < bj) {
          float2 r0 = acc2[bi * B + gq], r1 = acc2[bi * B + gq + 8];
          float d[4] = {r0.x, r0.y, r1.x, r1.y};
          M::mma(d, raw.x, raw.z, raw.y, raw.w, br.x, br.y);
          if (owner) {
            acc2[bi * B + gq] = make_float2(d[0], d[1]);
            acc2[bi * B + gq + 8] = make_float2(d[2], d[3]);
          }
        }
        const uint2 bc = bsrc[bi * 8];
        M::mma(dc, movm_trans(raw.x), movm_trans(raw.y), movm_trans(raw.z), movm_trans(raw.w), bc.x, bc.y);
      });
      // the column's sums: row block bj has taken no row part yet
      if (owner) {
        acc2[bj * B + kxq] = make_float2(dc[0], dc[1]);
        acc2[bj * B + kyq] = make_float2(dc[2], dc[3]);
      }
      __syncwarp();  // before later row parts read these from other lanes
    }
  });
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    if (s < p) {
      const float2 a = acc2[s];
      *reinterpret_cast<float2*>(cur + 2 * (size_t)(p0 + s)) = make_float2(w_in[s], cs[s] + (a.x + a.y) * isc);
    }
  }
  if (valid && lane == 0) partials2[(size_t)(k & 1) * nparts + dsc.tile] = (double)tile_sq * pow2d(2 * tile_e);
}

// ---------------------------------------------------------------------------
// FP64-accurate packed sweep in double-float arithmetic (kernel 12; plain
// FP64 plans of a symmetric A, tiles of at most 128 ports).  GB300 executes
// FP64 at about 2 FMA per clock per SM, so the FP64 sweeps of the full T_P
// (kernels 1-4) are bound by that pipe, not by HBM.  This kernel keeps FP64
// bytes (each stored entry of T_P is the pair hi = rn32(T), lo = rn32(T -
// hi), 8 bytes, about 48 significant bits; the waves and c are such pairs
// too) and does all arithmetic on the FP32 pipes with error-free
// transformations (df.cuh): the products of a block accumulate as in Dot2
// (high parts through TwoSum, every error term in a second FP32 word), the
// residual terms in double-word arithmetic.  Only the packed upper blocks are
// stored (T_P is symmetric for scalar W, Sec. VIII), half the bytes of the
// full FP64 matrix.
// Organisation of kernel 9: one warp per tile (one CTA per SM, four service
// warps of CTA 0 decide on the previous sweep, three wave slots, sweep
// number from the ticket), blocks column by column with a per-warp ring of
// KB asynchronously copied blocks.  A block is 2 KB: its hi block then its lo
// block, each in the FP32 layout (lane l reads float4 l and l + 32: rows l/4
// and l/4 + 8, columns 4(l%4)..+3).  State per port and slot: (w_in.h,
// w_in.l, w_out.h, w_out.l).
// ---------------------------------------------------------------------------

constexpr int kWdfKB = 2;  // ring slots per warp (2 KB each)

// per warp: the ring, then w_in and the output accumulators (the residual
// terms live in the last ring slot, which no copy fills before the blocks)
__host__ __device__ constexpr size_t wdf_warp_bytes(int pp_max, int kb) {
  return (size_t)kb * 2 * kSymB * kSymB * sizeof(float) + 16 * (size_t)pp_max;
}

__device__ __forceinline__ df shfl_xor_df(df v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.h, m), __shfl_xor_sync(0xffffffffu, v.l, m)};
}
__device__ __forceinline__ dacc shfl_xor_dacc(dacc v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.S, m), __shfl_xor_sync(0xffffffffu, v.E, m)};
}

// Residual term of a torn branch (port_residual above) in double-word
// arithmetic: the sum cancels to the residual, so every operation keeps
// about 44 bits of its operands, the coefficients (g/W, d) included (kq =
// (g/W hi, lo, d hi, lo)).
__device__ __forceinline__ df port_residual_df(df wi_s, df wo_s, df wi_t, df wo_t, float4 kq) {
  const df Ss = df_add(wi_s, wo_s), St = df_add(wi_t, wo_t);
  df a = df_add(Ss, St);
  a = {0.5f * a.h, 0.5f * a.l};
  const df gd = df_mul(df_sub(Ss, St), df{kq.x, kq.y});
  const df r = df_sub(df_sub(df_sub(a, gd), wi_s), wi_t);
  const df hd = {0.5f * kq.z, 0.5f * kq.w};
  return df_mul(r, hd);
}

template <int KB>
__global__ void __launch_bounds__(1024, 1) sweep_wdf_kernel(
    const float* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float4* __restrict__ kd,
    const uint8_t* __restrict__ run, const float2* __restrict__ c, float4* __restrict__ state3,
    int64_t nports, SweepCtrl* __restrict__ ctrl,
    double* __restrict__ partials2, double* __restrict__ hist, int hist_len, int nparts, int pp_max) {
  constexpr int B = kSymB;
  constexpr int PPL = 4;
  constexpr int BLK = 2 * B * B;  // floats of one stored block (hi, lo)
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_k, s_flag;
  __shared__ double s_red[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (int)(blockDim.x >> 5) - 4;  // tile warps; the last four serve
  if (tid == 0) s_flag = *((volatile int*)&ctrl->flag);
  __syncthreads();
  if (s_flag) return;
  const bool tile_warp = warp < nw;
  const int g = warp * gridDim.x + blockIdx.x;  // tiles dealt round the CTAs
  const bool valid = tile_warp && g < nparts;
  TileDesc dsc{};
  if (valid) dsc = tdesc[g];
  const int p0 = dsc.p0, p = valid ? dsc.p : 0;
  const int nb = (p + B - 1) / B;
  const int nblk = nb * (nb + 1) / 2;
  const float* Tl = Tp + 2 * dsc.Tp_off;
  float* ring = reinterpret_cast<float*>(smem_raw + (size_t)(tile_warp ? warp : 0) * wdf_warp_bytes(pp_max, KB));
  df* w_in = reinterpret_cast<df*>(ring + KB * BLK);
  dacc* acc = reinterpret_cast<dacc*>(w_in + pp_max);
  // residual terms: in ring slot KB - 1, free until the block loop's first copy
  df* rs = reinterpret_cast<df*>(ring + (KB - 1) * BLK);
  int tw[PPL];
  uint32_t rn4 = 0;
  int pbi = 0, pbj = 0, pidx = 0, pq = 0;
  auto issue_next = [&]() {
    if (pq < nblk) {
      float* dst = ring + (pq % KB) * BLK;
      const float* src = Tl + (size_t)pidx * BLK;
#pragma unroll
      for (int h = 0; h < 4; ++h) cp_async16(dst + 4 * (lane + 32 * h), src + 4 * (lane + 32 * h));
      if (pbi < pbj) {
        pidx += nb - 1 - pbi;
        ++pbi;
      } else {
        ++pbj;
        pbi = 0;
        pidx = pbj;
      }
    }
    ++pq;
    cp_async_commit_group();
  };
  if (tile_warp) {
#pragma unroll
    for (int b = 0; b < KB - 1; ++b) issue_next();
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      tw[m] = s < p ? twin[p0 + s] : 0;
      if (s < p) rn4 |= (uint32_t)run[p0 + s] << (8 * m);
    }
  }
  pdl_launch_dependents();
  pdl_wait();  // the previous sweep's waves, partials and decision
  if (tid == 0) {
    s_flag = *((volatile int*)&ctrl->flag);
    if (!s_flag) s_k = (int)take_sweep_number(ctrl);
  }
  __syncthreads();
  if (s_flag) {
    cp_async_wait_group<0>();  // no copy into shared memory outlives the CTA
    return;
  }
  const int k = s_k;
  if (!tile_warp) {  // service warps: CTA 0 decides on the previous sweep
    if (blockIdx.x != 0 || k < 2) return;
    const int t = tid - nw * 32;
    const double tot = group128_sum_fixed(partials2 + (size_t)((k - 1) & 1) * nparts, nparts, t, s_red);
    if (t == 0) sweep_decide(ctrl, k - 1, tot, hist, hist_len);
    return;
  }
  const float4* prev = state3 + (size_t)((k - 1) % 3) * nports;
  float4* cur = state3 + (size_t)(k % 3) * nports;
  // incident waves and residual terms of sweep k - 1; the outputs start at c
  {
    float2 c0v[PPL];
    float4 wtv[PPL], wsv[PPL], kqv[PPL];
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      c0v[m] = make_float2(0.f, 0.f);
      wtv[m] = wsv[m] = kqv[m] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s < p) {
        c0v[m] = c[p0 + s];
        if (k > 1) {
          wtv[m] = prev[tw[m]];
          wsv[m] = prev[p0 + s];
          kqv[m] = kd[p0 + s];
        }
      }
    }
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      if (s < nb * B) {
        df wi = {0.f, 0.f}, rc = {0.f, 0.f};
        if (s < p && k > 1) {
          wi = {wtv[m].z, wtv[m].w};  // the twin's outgoing wave
          rc = port_residual_df({wsv[m].x, wsv[m].y}, {wsv[m].z, wsv[m].w}, {wtv[m].x, wtv[m].y}, wi, kqv[m]);
        }
        w_in[s] = wi;
        rs[s] = rc;
        acc[s] = {c0v[m].x, c0v[m].y};
      }
    }
  }
  __syncwarp();
  df tile_sq = {0.f, 0.f};  // lane 0: the four groups in order, scaled by 2^-2 tile_e
  int tile_e = 0;
  if (k > 1) {
    df rrv[PPL];
    float rmax = 0.f;
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      const int nr = (rn4 >> (8 * m)) & 0xff;
      df rr = {0.f, 0.f};
      if (s < p && nr) {
        rr = rs[s];
        for (int q = 1; q < nr; ++q) rr = df_add(rr, rs[s + q]);
      }
      rrv[m] = rr;
      rmax = fmaxf(rmax, fabsf(rr.h));
    }
    tile_e = pow2_exponent(warp_max(rmax));
    const float rsc = pow2f(-tile_e);
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      df sq = {0.f, 0.f};
      const int s = lane + 32 * m;
      const int nr = (rn4 >> (8 * m)) & 0xff;
      if (s < p && nr) {
        const df rr = {rrv[m].h * rsc, rrv[m].l * rsc};
        sq = df_mul(rr, rr);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const df t = {__shfl_down_sync(FULL, sq.h, o), __shfl_down_sync(FULL, sq.l, o)};
        sq = df_add(sq, t);
      }
      tile_sq = df_add(tile_sq, sq);
    }
  }
  // Blocks in column-major order over the upper triangle, as in kernel 9:
  // each block's row partial is reduced at once into its row block; its
  // column partial accumulates in registers over the block column (four
  // columns x two rows per lane) and is reduced across the eight lanes of a
  // column group after the diagonal block.
  const int r1 = lane >> 2, cg = lane & 3;
  const bool b0 = lane & 1, b4 = lane & 16, b3 = lane & 8;
  const bool row_owner = !(lane & 2), col_owner = !(lane & 4);
  const int myrow = b0 ? r1 + 8 : r1;
  const int mycol = cg * 4 + (b4 ? 2 : 0) + (b3 ? 1 : 0);
  // column partials of columns (0, 1) and (2, 3) of this lane's four, as pairs
  dacc2 ca01 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, ca23 = ca01;
  int bi = 0, bj = 0;
  for (int kk = 0; kk < nblk; ++kk) {
    issue_next();
    cp_async_wait_group<KB - 1>();  // this lane's bytes of block kk have landed
    const float* blk = ring + (kk % KB) * BLK;
    const float4 ha = reinterpret_cast<const float4*>(blk)[lane];
    const float4 hb = reinterpret_cast<const float4*>(blk)[lane + 32];
    const float4 la = reinterpret_cast<const float4*>(blk + B * B)[lane];
    const float4 lb = reinterpret_cast<const float4*>(blk + B * B)[lane + 32];
    {  // row partials of rows r1 (a) and r1 + 8 (b) over this lane's four columns,
       // the two rows as the halves of one pair
      const df* wc = w_in + bj * B + cg * 4;
      const df w0 = wc[0], w1 = wc[1], w2 = wc[2], w3 = wc[3];
      dacc2 x = dacc2_first(make_float2(ha.x, hb.x), make_float2(la.x, lb.x), make_float2(w0.h, w0.h),
                            make_float2(w0.l, w0.l));
      dacc2_fma(x, make_float2(ha.y, hb.y), make_float2(la.y, lb.y), make_float2(w1.h, w1.h),
                make_float2(-w1.h, -w1.h), make_float2(w1.l, w1.l));
      dacc2_fma(x, make_float2(ha.z, hb.z), make_float2(la.z, lb.z), make_float2(w2.h, w2.h),
                make_float2(-w2.h, -w2.h), make_float2(w2.l, w2.l));
      dacc2_fma(x, make_float2(ha.w, hb.w), make_float2(la.w, lb.w), make_float2(w3.h, w3.h),
                make_float2(-w3.h, -w3.h), make_float2(w3.l, w3.l));
      const dacc x1 = dacc2_lo(x), x2 = dacc2_hi(x);
      // the row's four lanes (bits 0, 1): reduce-scatter over bit 0, sum over bit 1
      dacc t = dacc_add(b0 ? x2 : x1, shfl_xor_dacc(b0 ? x1 : x2, 1));
      t = dacc_add(t, shfl_xor_dacc(t, 2));
      if (row_owner) acc[bi * B + myrow] = dacc_add(acc[bi * B + myrow], t);
    }
    if (bi != bj) {
      // columns (0, 1) and (2, 3) as pairs, rows r1 and r1 + 8 one after the other
      const df wr1 = w_in[bi * B + r1], wr2 = w_in[bi * B + r1 + 8];
      const float2 h1 = make_float2(wr1.h, wr1.h), n1 = make_float2(-wr1.h, -wr1.h), l1 = make_float2(wr1.l, wr1.l);
      const float2 h2 = make_float2(wr2.h, wr2.h), n2 = make_float2(-wr2.h, -wr2.h), l2 = make_float2(wr2.l, wr2.l);
      dacc2_fma(ca01, make_float2(ha.x, ha.y), make_float2(la.x, la.y), h1, n1, l1);
      dacc2_fma(ca01, make_float2(hb.x, hb.y), make_float2(lb.x, lb.y), h2, n2, l2);
      dacc2_fma(ca23, make_float2(ha.z, ha.w), make_float2(la.z, la.w), h1, n1, l1);
      dacc2_fma(ca23, make_float2(hb.z, hb.w), make_float2(lb.z, lb.w), h2, n2, l2);
      ++bi;
    } else {
      __syncwarp();  // the diagonal block's row partial is in before the column's
      if (bj > 0) {
        // columns 4 cg..+3: sums over the eight lanes of a column group (bits 4, 3, 2)
        const dacc c0 = dacc2_lo(ca01), c1 = dacc2_hi(ca01), c2 = dacc2_lo(ca23), c3 = dacc2_hi(ca23);
        dacc k0 = b4 ? c2 : c0, k1 = b4 ? c3 : c1;
        k0 = dacc_add(k0, shfl_xor_dacc(b4 ? c0 : c2, 16));
        k1 = dacc_add(k1, shfl_xor_dacc(b4 ? c1 : c3, 16));
        dacc t1 = dacc_add(b3 ? k1 : k0, shfl_xor_dacc(b3 ? k0 : k1, 8));
        t1 = dacc_add(t1, shfl_xor_dacc(t1, 4));
        if (col_owner) acc[bj * B + mycol] = dacc_add(acc[bj * B + mycol], t1);
      }
      __syncwarp();  // and the column partial before later rows add to this block
      ca01 = ca23 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      ++bj;
      bi = 0;
    }
  }
  cp_async_wait_group<0>();
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    if (s < p) {
      const df o = dacc_value(acc[s]);
      cur[p0 + s] = make_float4(w_in[s].h, w_in[s].l, o.h, o.l);
    }
  }
  if (valid && lane == 0)
    partials2[(size_t)(k & 1) * nparts + dsc.tile] = ((double)tile_sq.h + (double)tile_sq.l) * pow2d(2 * tile_e);
}

// c as double-float pairs (once per inner solve of kernel 12)
__global__ void split_df_kernel(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i];
    const float h = (float)v;
    b[i] = make_float2(h, (float)(v - (double)h));
  }
}

// the chosen double-float wave slot as FP64 (w_in, w_out) pairs for the
// recovery
__global__ void join_df_kernel(const float4* __restrict__ st, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = st[i];
    out[2 * i] = (double)v.x + (double)v.y;
    out[2 * i + 1] = (double)v.z + (double)v.w;
  }
}

// ---------------------------------------------------------------------------
// Dataflow sweeps: one cooperative launch runs every sweep of an inner solve.
// Sweep k of tile P needs only the sweep-(k-1) waves of the tiles across its
// lines (the one-sweep delay of Eq. 11), so instead of a kernel boundary per
// sweep each tile waits for its neighbours' done counters.  The iterates are
// those of the launch-per-sweep kernels (same arithmetic, packed blocks).
//   * waves live in three slots (sweep k writes slot k mod 3): a tile may run
//     one sweep ahead of a neighbour, and the slot of the converged iterate
//     must survive the sweep after it;
//   * the last tile to finish sweep k reduces the residual partials of sweep
//     k (slot k mod 4, fixed order) and publishes the decision (gk = k); no
//     tile starts sweep k + 2 before that, so a stop decided at sweep k never
//     meets a tile that has overwritten what the host recovers from;
//   * every wait is bounded; a wait that runs out sets flag 5 (VTM_ETIMEOUT)
//     and any wait returns as soon as a flag is set.
// All CTAs are co-resident (cooperative launch), so the waits always end.
// ---------------------------------------------------------------------------

// A wait gives up after `max_polls` polls (vtm_opts.wait_polls; default 2^22,
// a few seconds).  lag_sel < 0 (vtm_opts.flow_lag = -1) makes every tile
// wait for the decision of its own sweep, which needs that very sweep: a
// host-made hang that the bounded waits must end (VTM_ETIMEOUT).

// Warp 0 waits (bounded) until the published decision has reached sweep
// k - 2 and every tile across the lines of `tile` has finished sweep k - 1:
// its lanes read the counters at once (lane 31 the decision, lanes 0..30 a
// chunk of neighbours).  false if a flag is raised (or the wait ran out, and
// then flag 5 is set).  Called by all 32 lanes of warp 0.
__device__ __forceinline__ bool flow_wait_ready(const int* gk, const int* done,
                                                const int32_t* __restrict__ nbr, int e0, int e1, int k,
                                                SweepCtrl* ctrl, uint32_t max_polls, int lag = 2) {
  const int lane = threadIdx.x & 31;
  for (int base = e0; base < e1 || base == e0; base += 31) {
    const int e = base + lane;
    const int* p = lane == 31 ? gk : (e < e1 ? done + nbr[e] : nullptr);
    const int need = lane == 31 ? k - lag : k - 1;
    uint32_t i = 0;
    for (;; ++i) {
      const bool ok = !p || *((volatile const int*)p) >= need;
      if (__all_sync(0xffffffffu, ok)) break;
      if (i >= max_polls) {
        if (lane == 0) atomicCAS(&ctrl->flag, 0, 5);
        return false;
      }
      if ((i & 15u) == 15u && *((volatile int*)&ctrl->flag)) return false;
      // back off: a spinning warp takes issue slots from the warps that work
      if (i >= 2) __nanosleep(i < 16 ? 64 : 256);
    }
  }
  return true;
}

// ASYNC: asynchronous VTM (Sec. XI: lines with different, varying delays).
// No neighbour waits and one wave slot: a tile reads whatever waves its
// neighbours last wrote (delay 0, 1 or 2 sweeps; the decision lag still keeps
// every tile within two sweeps of the slowest).  The fixed point is the same;
// the iterates depend on timing.
template <class TT, int NT, int KB, bool ASYNC>
__global__ void __launch_bounds__(NT, 768 / NT) sweep_flow_kernel(
    const TT* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state3,
    int64_t nports, const int32_t* __restrict__ nbr_off, const int32_t* __restrict__ nbr,
    int* __restrict__ done, unsigned* __restrict__ count, int* __restrict__ gk,
    SweepCtrl* __restrict__ ctrl, double* __restrict__ part4, double* __restrict__ hist,
    int hist_len, int nparts, int pp_max, int k0, uint32_t max_polls, int lag_sel) {
  using LD = SymLoad<TT>;
  constexpr int NW = NT / 32;
  constexpr int B = kSymB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_stop;
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* w_in = reinterpret_cast<float*>(smem_raw);
  float* rs = w_in + pp_max;
  float* part = rs + pp_max;
  for (int k = k0;; ++k) {
    for (int slot = blockIdx.x; slot < nparts; slot += gridDim.x) {
      const TileDesc dsc = tdesc[slot];
      const int tile = dsc.tile, p0 = dsc.p0, p = dsc.p;
      const int nb = (p + B - 1) / B;
      const int nblk = nb * (nb + 1) / 2;
      const TT* Tl = Tp + dsc.Tp_off;
      // what does not depend on the waves goes out before the waits
      typename LD::raw buf[KB];
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const int kk = warp + b * NW;
        if (kk < nblk) buf[b] = LD::load(Tl + (size_t)kk * B * B, lane);
      }
      SymPorts<NT> pt;
      pt.load(twin, kd, run, c, p0, p);
      if (warp == 0) {
        const int wlag = lag_sel < 0 ? 0 : 2;
        bool ok = ASYNC ? flow_wait_ready(gk, done, nbr, 0, 0, k, ctrl, max_polls, wlag)
                        : flow_wait_ready(gk, done, nbr, nbr_off[tile], nbr_off[tile + 1], k, ctrl, max_polls,
                                          wlag);
        __threadfence();  // every lane that saw a counter orders its later reads
        if (tid == 0) s_stop = (ok && !*((volatile int*)&ctrl->flag)) ? 0 : 1;
      }
      __syncthreads();
      if (s_stop) return;
      const float* prev = state3 + (ASYNC ? 0 : (size_t)((k - 1) % 3) * nports * 2);
      float* cur = state3 + (ASYNC ? 0 : (size_t)(k % 3) * nports * 2);
      const float sq = sym_gather<NT>(pt, prev, w_in, rs, p0, p, nb, k);
      const double tile_sq = (double)block_sum_value_f(sq);
      int bi = 0, off = warp;
      for (int base = 0; base < nblk; base += KB * NW) {
#pragma unroll
        for (int b = 0; b < KB; ++b) {
          const int kk = warp + base + b * NW;
          if (kk < nblk) {
            while (off >= nb - bi) {
              off -= nb - bi;
              ++bi;
            }
            const typename LD::raw v = buf[b];
            const int kn = kk + KB * NW;
            if (kn < nblk) buf[b] = LD::load(Tl + (size_t)kn * B * B, lane);
            sym_apply<TT>(v, bi, bi + off, lane, w_in, PartSink{part, nb});
            off += NW;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < SymPorts<NT>::PPT; ++j) {
        const int s = tid + j * NT;
        if (s < p) {
          const int a = s / B, rr = s % B;
          float acc = pt.cq[j];
          for (int b = 0; b < nb; ++b) acc += part[(a * nb + b) * B + rr];
          *reinterpret_cast<float2*>(cur + 2 * (size_t)(p0 + s)) = make_float2(w_in[s], acc);
        }
      }
      __threadfence();  // this thread's waves are visible device-wide before the done counter moves
      __syncthreads();
      if (tid == 0) {
        part4[(size_t)(k & 3) * nparts + tile] = tile_sq;
        __threadfence();
        atomicExch(done + tile, k);
        s_last = atomicAdd(count + (k & 3), 1u) == (unsigned)nparts - 1;
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        const double tot = block_sum_fixed(part4 + (size_t)(k & 3) * nparts, nparts);
        if (tid == 0) {
          sweep_decide(ctrl, k, tot, hist, hist_len);
          count[(k + 2) & 3] = 0u;
          __threadfence();
          atomicExch(gk, k);
        }
        __syncthreads();
      }
    }
  }
}

// Dataflow sweeps with one warp per tile (every tile resident: one warp each,
// kWflowWarps per CTA, a cooperative launch per inner solve).  Each warp runs
// the sweeps of its own tile: it waits (flow_wait_ready) until the tiles
// across its lines have finished sweep k - 1 and the published decision has
// reached sweep k - 2, then gathers, streams its blocks and publishes its done
// counter.  The tile's blocks are the same for every sweep, so its cp.async
// ring runs on across sweep boundaries: the blocks of sweep k + 1 are in
// flight while the warp publishes sweep k and waits for its neighbours.
// Waves live in three slots, as for sweep_flow_kernel.  The residual of sweep
// k - 1 (computed in sweep k) is reduced in two fixed-order levels off the
// critical path: the last tile of each group of G tiles sums the group's
// partials, the last group sums the group sums and publishes the decision.
// Block arithmetic and order are those of kernel 9, blocks column by column
// (the iterates match it bitwise; the residual sums differ by their order
// only).  Asynchronous VTM runs it with a decision lag of 8 (kLag).
template <class TT, int KB, bool ASYNC>
__global__ void __launch_bounds__(32 * kWflowWarps, kWflowCtasPerSm) sweep_wflow_kernel(
    const TT* __restrict__ Tp, const TileDesc* __restrict__ tdesc,
    const int32_t* __restrict__ twin, const float2* __restrict__ kd,
    const uint8_t* __restrict__ run, const float* __restrict__ c, float* __restrict__ state3,
    int64_t nports, const int32_t* __restrict__ nbr_off, const int32_t* __restrict__ nbr,
    int* __restrict__ done, unsigned* __restrict__ count, int* __restrict__ gk,
    unsigned* __restrict__ gcount, double* __restrict__ gsum, int G,
    SweepCtrl* __restrict__ ctrl, double* __restrict__ part4, double* __restrict__ hist,
    int hist_len, int nparts, int pp_max, int k0, uint32_t max_polls, int lag_sel) {
  using LD = SymLoad<TT>;
  constexpr int B = kSymB;
  constexpr int PPL = 4;
  // decision lag: a tile starts sweep k once the decision of sweep k - kLag is
  // out.  Synchronous sweeps keep their three wave slots safe with 2; the
  // asynchronous iteration has one slot and runs ahead by up to 8.  Counters
  // and partials of the sweeps in flight live in kSlots ring entries.
  constexpr int kLag = ASYNC ? 8 : 2;
  constexpr int kSlots = 16;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = blockIdx.x * kWflowWarps + warp;
  if (g >= nparts) return;  // no CTA barrier below: idle warps just leave
  const TileDesc dsc = tdesc[g];
  const int tile = dsc.tile, p0 = dsc.p0, p = dsc.p;
  const int nb = (p + B - 1) / B;
  const int nblk = nb * (nb + 1) / 2;
  const TT* Tl = Tp + dsc.Tp_off;
  TT* ring = reinterpret_cast<TT*>(smem_raw + (size_t)warp * (KB * B * B * sizeof(TT) + 12 * (size_t)pp_max));
  float* w_in = reinterpret_cast<float*>(ring + KB * B * B);
  float* rs = w_in + pp_max;
  float* acc = rs + pp_max;
  const int ngroups = (nparts + G - 1) / G;
  const int grp = g / G;
  const unsigned gsize = (unsigned)min(G, nparts - grp * G);
  const int e0 = ASYNC ? 0 : nbr_off[tile], e1 = ASYNC ? 0 : nbr_off[tile + 1];
  int tw[PPL];
  uint32_t rn4 = 0;
#pragma unroll
  for (int m = 0; m < PPL; ++m) {
    const int s = lane + 32 * m;
    tw[m] = s < p ? twin[p0 + s] : 0;
    if (s < p) rn4 |= (uint32_t)run[p0 + s] << (8 * m);
  }
  // the block stream of the tile repeats every sweep, in the column-major
  // order of sweep_wsym_kernel: copy number qn goes to ring slot qn mod KB and
  // is block (pbi, pbj), number pidx of the row-major packed tile
  int q = 0, qn = 0, pbi = 0, pbj = 0, pidx = 0;
  auto issue = [&]() {
    if (nblk) {
      copy_block_async(ring + (qn % KB) * B * B, Tl + (size_t)pidx * B * B, lane);
      if (pbi < pbj) {
        pidx += nb - 1 - pbi;
        ++pbi;
      } else if (pbj + 1 < nb) {
        ++pbj;
        pbi = 0;
        pidx = pbj;
      } else {
        pbi = pbj = pidx = 0;  // the next sweep's first block
      }
    }
    cp_async_commit_group();
    ++qn;
  };
#pragma unroll
  for (int b = 0; b < KB - 1; ++b) issue();
  const int r1 = lane >> 2, cg = lane & 3;
  const bool b0 = lane & 1, b4 = lane & 16, b3 = lane & 8;
  const bool row_owner = !(lane & 2), col_owner = !(lane & 4);
  const int myrow = b0 ? r1 + 8 : r1;
  const int mycol = cg * 4 + (b4 ? 2 : 0) + (b3 ? 1 : 0);
  for (int k = k0;; ++k) {
    const bool ok = flow_wait_ready(gk, done, nbr, e0, e1, k, ctrl, max_polls, lag_sel < 0 ? 0 : kLag);
    __threadfence();  // every lane that saw a counter orders its later reads
    int stop = 0;
    if (lane == 0) stop = (ok && !*((volatile int*)&ctrl->flag)) ? 0 : 1;
    if (__shfl_sync(FULL, stop, 0)) {
      cp_async_wait_group<0>();  // no copy into shared memory outlives the warp
      return;
    }
    const float* prev = state3 + (ASYNC ? 0 : (size_t)((k - 1) % 3) * nports * 2);
    float* cur = state3 + (ASYNC ? 0 : (size_t)(k % 3) * nports * 2);
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      if (s < nb * B) {
        float wi = 0.f, rc = 0.f, c0 = 0.f;
        if (s < p) {
          c0 = c[p0 + s];
          if (k > 1) {
            const float2 wt = __ldcg(reinterpret_cast<const float2*>(prev + 2 * (size_t)tw[m]));
            const float2 ws = __ldcg(reinterpret_cast<const float2*>(prev + 2 * (size_t)(p0 + s)));
            wi = wt.y;
            rc = port_residual<float>(ws.x, ws.y, wt.x, wt.y, kd[p0 + s]);
          }
        }
        w_in[s] = wi;
        rs[s] = rc;
        acc[s] = c0;
      }
    }
    __syncwarp();
    float tile_sq = 0.f;
    if (k > 1) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float sq = 0.f;
        const int s = lane + 32 * v;
        const int nr = (rn4 >> (8 * v)) & 0xff;
        if (s < p && nr) {
          float rr = 0.f;
          for (int qq = 0; qq < nr; ++qq) rr += rs[s + qq];
          sq += rr * rr;
        }
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(FULL, sq, o);
        tile_sq += sq;
      }
    }
    // blocks column by column, as in sweep_wsym_kernel (the same arithmetic)
    float2 ca01 = make_float2(0.f, 0.f), ca23 = make_float2(0.f, 0.f);
    int bi = 0, bj = 0;
    for (int kk = 0; kk < nblk; ++kk, ++q) {
      issue();  // stream number q + KB - 1
      cp_async_wait_group<KB - 1>();  // this lane's bytes of block kk have landed
      SymLoad<float>::raw v;
      if constexpr (std::is_same<TT, float>::value) {
        v = LD::load_shared(ring + (q % KB) * B * B, lane);
      } else {
        const uint4 raw = LD::load_shared(ring + (q % KB) * B * B, lane);
        const float2 e0_ = Pair16<TT>::f2(raw.x), e1_ = Pair16<TT>::f2(raw.y);
        const float2 e2_ = Pair16<TT>::f2(raw.z), e3_ = Pair16<TT>::f2(raw.w);
        v.a = make_float4(e0_.x, e0_.y, e1_.x, e1_.y);
        v.b = make_float4(e2_.x, e2_.y, e3_.x, e3_.y);
      }
      const float2 a01 = make_float2(v.a.x, v.a.y), a23 = make_float2(v.a.z, v.a.w);
      const float2 b01 = make_float2(v.b.x, v.b.y), b23 = make_float2(v.b.z, v.b.w);
      {
        const float4 wc = *reinterpret_cast<const float4*>(w_in + bj * B + cg * 4);
        const float2 wc01 = make_float2(wc.x, wc.y), wc23 = make_float2(wc.z, wc.w);
        const float2 pa = __ffma2_rn(a23, wc23, __fmul2_rn(a01, wc01));
        const float2 pb = __ffma2_rn(b23, wc23, __fmul2_rn(b01, wc01));
        const float x1 = pa.x + pa.y, x2 = pb.x + pb.y;
        float t = (b0 ? x2 : x1) + __shfl_xor_sync(FULL, b0 ? x1 : x2, 1);
        t += __shfl_xor_sync(FULL, t, 2);
        if (row_owner) acc[bi * B + myrow] += t;
      }
      if (bi != bj) {
        const float wr1 = w_in[bi * B + r1], wr2 = w_in[bi * B + r1 + 8];
        const float2 w1 = make_float2(wr1, wr1), w2 = make_float2(wr2, wr2);
        ca01 = __ffma2_rn(b01, w2, __ffma2_rn(a01, w1, ca01));
        ca23 = __ffma2_rn(b23, w2, __ffma2_rn(a23, w1, ca23));
        ++bi;
      } else {
        __syncwarp();
        if (bj > 0) {
          float k0 = b4 ? ca23.x : ca01.x, k1 = b4 ? ca23.y : ca01.y;
          k0 += __shfl_xor_sync(FULL, b4 ? ca01.x : ca23.x, 16);
          k1 += __shfl_xor_sync(FULL, b4 ? ca01.y : ca23.y, 16);
          float t1 = (b3 ? k1 : k0) + __shfl_xor_sync(FULL, b3 ? k0 : k1, 8);
          t1 += __shfl_xor_sync(FULL, t1, 4);
          if (col_owner) acc[bj * B + mycol] += t1;
        }
        __syncwarp();
        ca01 = ca23 = make_float2(0.f, 0.f);
        ++bj;
        bi = 0;
      }
    }
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
      const int s = lane + 32 * m;
      if (s < p) *reinterpret_cast<float2*>(cur + 2 * (size_t)(p0 + s)) = make_float2(w_in[s], acc[s]);
    }
    // publish: partial, done counter, then the two-level residual sum (every
    // lane's waves are visible device-wide before the done counter moves)
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) {
      part4[(size_t)(k & (kSlots - 1)) * nparts + g] = (double)tile_sq;
      __threadfence();
      atomicExch(done + tile, k);
      last = atomicAdd(gcount + (k & (kSlots - 1)) * 32 + grp, 1u) == gsize - 1;
    }
    if (__shfl_sync(FULL, last, 0)) {
      __threadfence();
      const double* pg = part4 + (size_t)(k & (kSlots - 1)) * nparts + (size_t)grp * G;
      double s = 0.0;
      for (int i = lane; i < (int)gsize; i += 32) s += __ldcg(pg + i);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(FULL, s, o);
      int top = 0;
      if (lane == 0) {
        gsum[(k & (kSlots - 1)) * 32 + grp] = s;
        __threadfence();
        top = atomicAdd(count + (k & (kSlots - 1)), 1u) == (unsigned)ngroups - 1;
      }
      if (__shfl_sync(FULL, top, 0)) {
        __threadfence();
        double t = lane < ngroups ? __ldcg(gsum + (k & (kSlots - 1)) * 32 + lane) : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(FULL, t, o);
        // counters of sweep k + 2 start from zero before anyone may finish it
        gcount[((k + kLag) & (kSlots - 1)) * 32 + lane] = 0u;
        __threadfence();
        __syncwarp();
        if (lane == 0) {
          count[(k + kLag) & (kSlots - 1)] = 0u;
          sweep_decide(ctrl, k, t, hist, hist_len);
          __threadfence();
          atomicExch(gk, k);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

static int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

struct SweepLaunch {
  const void* T;
  const void* c;
  void* state;
  int prec;
};

// per-port residual coefficients (g/W, d) in the wave precision
template <class WT>
static const typename KdOf<WT>::type* kd_of(vtm_plan_s* P) {
  if constexpr (std::is_same<WT, double>::value) return P->d_kd.as<double2>();
  else return P->d_kd32.as<float2>();
}

// One launch of a packed sweep (kernels 5-7), as a programmatic dependent of
// the kernel before it on the stream unless the plan turned that off
// (vtm_opts.pdl = 1).  Launch errors surface through cudaGetLastError.
template <class... KArgs, class... Args>
static void launch_packed(const vtm_plan_s* P, void (*kern)(KArgs...), int grid, int threads, size_t smem,
                          cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = P->opts.pdl == 1 ? 0 : 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <class TT, class WT>
static void launch_sweep(vtm_plan_s* P, const TT* T, const WT* c, WT* state, int threads,
                         size_t smem, double* hist, int hist_len) {
  sweep_kernel<TT, WT><<<P->nparts, threads, smem, P->stream>>>(
      T, P->tabs.T_off.as<int64_t>(), P->tabs.T_ld.as<int32_t>(), P->tabs.port_off.as<int32_t>(),
      P->tabs.order.as<int32_t>(), P->d_twin.as<int32_t>(), kd_of<WT>(P), P->d_run.as<uint8_t>(), c,
      state, (int64_t)P->port_node.size(), P->d_ctrl.as<SweepCtrl>(), P->d_partials.as<double>(), hist,
      hist_len, P->nparts);
}

// Scoped access-policy window on the plan's stream over the FP32/16-bit
// reflection matrices (their packed copy where the plan has one): a persisting L2 carve-out of up to the device's
// maximum is requested for this context and released (with the stream
// attribute and the previous limit) when the sweeps end.
struct L2Window {
  cudaStream_t s = nullptr;
  size_t old_limit = 0;
  bool active = false;
  L2Window(vtm_plan_s* P, int prec) {
    if (prec == VTM_PREC_FP64 || P->opts.l2_persist != 1 || !P->stream) return;
    // the packed copy when there is one (the packed kernels read only that)
    const DevBuf& full = prec == VTM_PREC_FP32 ? P->d_T32 : P->d_T16;
    const DevBuf& packed = prec == VTM_PREC_FP32 ? P->d_Tp32 : P->d_Tp16;
    const void* base = packed.p ? packed.p : full.p;
    const size_t bytes = packed.p ? packed.bytes : full.bytes;
    int maxp = 0, maxw = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, P->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, P->device) != cudaSuccess ||
        maxp <= 0 || maxw <= 0 || !base) {
      cudaGetLastError();
      return;
    }
    if (cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    const size_t carve = std::min<size_t>((size_t)maxp, bytes);
    const size_t win = std::min<size_t>((size_t)maxw, bytes);
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, carve) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaStreamAttrValue a{};
    a.accessPolicyWindow.base_ptr = const_cast<void*>(base);
    a.accessPolicyWindow.num_bytes = win;
    a.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)carve / (double)win);
    a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(P->stream, cudaStreamAttributeAccessPolicyWindow, &a) != cudaSuccess) {
      cudaGetLastError();
      cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
      return;
    }
    s = P->stream;
    active = true;
  }
  ~L2Window() {
    if (!active) return;
    cudaStreamAttrValue a{};
    a.accessPolicyWindow.num_bytes = 0;
    cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &a);
    cudaStreamSynchronize(s);
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
    cudaGetLastError();
  }
};

// Run sweeps from a zero state until the interface residual is below
// target2 (absolute, squared) or the sweep budget is used.  Returns the
// sweep whose waves are to be recovered and its flag.
// *P->h_ctrl to the device, with the per-CTA sweep counters zeroed
static vtm_status upload_ctrl(vtm_plan_s* P, cudaStream_t s) {
  VTM_CUDA_TRY(cudaMemcpyAsync(P->d_ctrl.p, P->h_ctrl, sizeof(SweepCtrl), cudaMemcpyHostToDevice, s));
  VTM_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<SweepCtrl*>(P->d_ctrl.p) + 1, 0,
                               P->d_ctrl.bytes - sizeof(SweepCtrl), s));
  return VTM_OK;
}

static vtm_status run_sweeps(vtm_plan_s* P, double bnorm2, double target2, int budget, int prec,
                             double* hist, int hist_len, int stall, int* sweep_out, int* flag_out,
                             int hint = 0) {
  cudaStream_t s = P->stream;
  const int64_t npt = (int64_t)P->port_node.size();
  SweepCtrl h{};
  h.k = 1;
  h.flag = 0;
  h.counter = 0;
  h.conv_sweep = 0;
  h.k_max = budget;
  h.stall = stall;
  h.best_k = 0;
  h.best_res2 = 0.0;
  h.tol2 = target2;
  h.bnorm2 = bnorm2 > 0 ? bnorm2 : 1.0;
  *P->h_ctrl = h;
  VTM_TRY(upload_ctrl(P, s));
  const int threads = P->max_ports <= 64 ? 64 : (P->max_ports <= 128 ? 128 : 256);
  size_t wsz = prec == VTM_PREC_FP64 ? sizeof(double) : sizeof(float);
  size_t smem = (size_t)((P->max_ports + 2) & ~1) * wsz * 2 + 16;
  if (prec == VTM_PREC_FP64) {
    VTM_CUDA_TRY(cudaMemsetAsync(P->d_state64.p, 0, 4 * npt * sizeof(double), s));
  } else {
    VTM_CUDA_TRY(cudaMemsetAsync(P->d_state32.p, 0, 4 * npt * sizeof(float), s));
  }
  // staged kernel: ring of kStages stages of `ch` rows, at most 16 KB per stage
  int ld_max = 8;
  for (int32_t v : P->T_ld) ld_max = std::max(ld_max, v);
  const size_t s_t = prec == VTM_PREC_FP64 ? 8 : (prec == VTM_PREC_FP32 ? 4 : 2);
  const int vec = prec == VTM_PREC_FP64 ? 2 : (prec == VTM_PREC_FP32 ? 4 : 8);
  int ch = (int)std::max<size_t>(1, (16 * 1024) / (ld_max * s_t));
  ch = std::min(ch, std::max(1, P->max_ports));
  const size_t st_smem = kStages * (size_t)ch * ld_max * s_t + 2 * (size_t)ld_max * wsz +
                         256 * (size_t)vec * wsz + 128;
  const int nv_max = (P->max_ports + vec - 1) / vec;
  // auto: the FP64 sweep is bound by GB300's FP64 pipe, where the direct-load
  // kernel does best; FP32/BF16/FP16 stream their matrices through the bulk-copy ring
  const int choice = P->opts.sweep_kernel
                         ? P->opts.sweep_kernel
                         : (prec == VTM_PREC_FP64 ? 1 : (nv_max <= 256 ? 3 : 2));
  const bool staged = choice == 2 && nv_max <= 4 * 256 && st_smem <= 200 * 1024;
  // vector-load kernel: every thread owns one vector column (nv <= threads)
  const bool vecload = (choice == 3 && nv_max <= 256) || (choice == 4 && nv_max <= 128);
  const size_t vec_smem = 2 * (size_t)ld_max * wsz + 256 * (size_t)vec * wsz + 16;
  // packed symmetric kernel (FP32/16-bit copies exist only for symmetric plans)
  const bool sym_ok = prec == VTM_PREC_FP32 ? P->d_Tp32.p != nullptr
                      : prec != VTM_PREC_FP64 ? P->d_Tp16.p != nullptr
                                              : false;
  // the 16-bit storage type of a BF16 or FP16 plan, as a tag for the launches
  auto with16 = [&](auto fn) {
    if (prec == VTM_PREC_FP16) fn(__half{});
    else fn(__nv_bfloat16{});
  };
  auto pick16 = [&](const void* bf16_kernel, const void* fp16_kernel) {
    return prec == VTM_PREC_FP16 ? fp16_kernel : bf16_kernel;
  };
  const void* staged_kfn =
      prec == VTM_PREC_FP64   ? (const void*)sweep_staged_kernel<double, double, 2, 4>
      : prec == VTM_PREC_FP32 ? (const void*)sweep_staged_kernel<float, float, 4, 4>
                              : pick16((const void*)sweep_staged_kernel<__nv_bfloat16, float, 8, 4>,
                                       (const void*)sweep_staged_kernel<__half, float, 8, 4>);
  const int pp_max = std::max(kSymB, (P->max_ports + kSymB - 1) / kSymB * kSymB);
  const int nb_max = pp_max / kSymB;
  const size_t sym_smem = (2 * (size_t)pp_max + (size_t)nb_max * nb_max * kSymB) * sizeof(float) + 16;
  // bulk-copy variant: the largest packed tile plus the same work arrays
  const int tbuf_elems = nb_max * (nb_max + 1) / 2 * kSymB * kSymB;
  const size_t symb_smem = (size_t)tbuf_elems * (prec == VTM_PREC_FP32 ? 4 : 2) + sym_smem;
  const bool symb_ok = sym_ok && symb_smem <= 160 * 1024;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  // one warp per tile: per warp a ring of blocks, w_in, residual terms and
  // outputs of the tile.  One CTA per SM holds ceil(nparts / SMs) tile warps
  // (at most 28, and what shared memory holds) and four service warps, so
  // every SM carries the same number of tiles; the variant for this
  // precision and tile size
  const size_t wsym_per_warp =
      (size_t)(prec == VTM_PREC_FP32 ? kWsymKB32 * 4 : kWsymKB16 * 2) * kSymB * kSymB + 12 * (size_t)pp_max;
  int wsym_warps = std::min(28, std::max(1, (P->nparts + sms - 1) / sms));
  wsym_warps = std::max(1, std::min(wsym_warps, (int)(220 * 1024 / wsym_per_warp)));
  const int wsym_grid = (P->nparts + wsym_warps - 1) / wsym_warps;
  const int wsym_threads = 32 * (wsym_warps + 4);
  const size_t wsym_smem = wsym_warps * wsym_per_warp;
  const size_t wflow_smem = kWflowWarps * wsym_per_warp;
  // kernel 11 (tensor-core block products): 16-bit blocks, at most 128 ports
  // per tile; per warp w_in, residual terms, c, (hi, lo) sums, B operands
  const bool wmma_ok = sym_ok && prec != VTM_PREC_FP32 && pp_max <= kWmmaNB * kSymB;
  const size_t wmma_per_warp = 20 * (size_t)pp_max + 128 * kWmmaNB;
  int wmma_warps = std::min(28, std::max(1, (P->nparts + sms - 1) / sms));
  wmma_warps = std::max(1, std::min(wmma_warps, (int)(220 * 1024 / wmma_per_warp)));
  const int wmma_grid = (P->nparts + wmma_warps - 1) / wmma_warps;
  const int wmma_threads = 32 * (wmma_warps + 4);
  const size_t wmma_smem = wmma_warps * wmma_per_warp;
  // kernel 12 (double-float FP64-accurate sweep): FP64 plans with the packed
  // double-float copy, at most 128 ports per tile
  const bool wdf_ok = prec == VTM_PREC_FP64 && P->d_Tpdf.p != nullptr && pp_max <= 8 * kSymB;
  const size_t wdf_per_warp = wdf_warp_bytes(pp_max, kWdfKB);
  int wdf_warps = std::min(28, std::max(1, (P->nparts + sms - 1) / sms));
  wdf_warps = std::max(1, std::min(wdf_warps, (int)(220 * 1024 / wdf_per_warp)));
  const int wdf_grid = (P->nparts + wdf_warps - 1) / wdf_warps;
  const int wdf_threads = 32 * (wdf_warps + 4);
  const size_t wdf_smem = wdf_warps * wdf_per_warp;
  if (wdf_ok) {
    VTM_TRY(dev_alloc(P->d_dfstate, 3 * (size_t)std::max<int64_t>(npt, 1) * sizeof(float4)));
    VTM_TRY(dev_alloc(P->d_cdf, (size_t)std::max<int64_t>(npt, 1) * sizeof(float2)));
    split_df_kernel<<<grid_for(std::max<int64_t>(npt, 1)), 256, 0, s>>>(P->d_c64.as<double>(),
                                                                        P->d_cdf.as<float2>(), npt);
    VTM_CUDA_TRY(cudaGetLastError());
    P->launch_count++;
    VTM_CUDA_TRY(cudaFuncSetAttribute(sweep_wdf_kernel<kWdfKB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)wdf_smem));
  }
  auto with_wsym = [&](auto fn) {
    const bool wide = pp_max > 128;
    if (prec == VTM_PREC_FP32) {
      if (wide) fn(sweep_wsym_kernel<float, kWsymKB32, 8>, P->d_Tp32.as<float>());
      else fn(sweep_wsym_kernel<float, kWsymKB32, 4>, P->d_Tp32.as<float>());
    } else {
      with16([&](auto h) {
        using H = decltype(h);
        if (wide) fn(sweep_wsym_kernel<H, kWsymKB16, 8>, P->d_Tp16.as<H>());
        else fn(sweep_wsym_kernel<H, kWsymKB16, 4>, P->d_Tp16.as<H>());
      });
    }
  };

  if (staged)
    VTM_CUDA_TRY(cudaFuncSetAttribute(staged_kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st_smem));
  const int st_threads = 256;
  const int64_t npt_ = npt;
  int st_grid = 0;
  auto launch_staged = [&](auto* kern, const auto* T, const auto* c, auto* state) {
    if (!st_grid) {
      int per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, st_threads, st_smem);
      st_grid = std::max(1, std::min(P->nparts, std::max(per_sm, 1) * sms));
    }
    kern<<<st_grid, st_threads, st_smem, s>>>(
        T, P->tabs.T_off.as<int64_t>(), P->tabs.T_ld.as<int32_t>(), P->tabs.port_off.as<int32_t>(),
        P->tabs.order.as<int32_t>(), P->d_twin.as<int32_t>(),
        kd_of<std::remove_pointer_t<decltype(state)>>(P), P->d_run.as<uint8_t>(), c, state, npt_,
        P->d_ctrl.as<SweepCtrl>(), P->d_partials.as<double>(), hist, hist_len, P->nparts, ch, ld_max);
  };
  // keep as much of the low-precision reflection matrices in L2 as the
  // persisting carve-out allows (restored after the sweeps)
  L2Window l2win(P, prec);
  // one sweep launch with kernel `kc` (1 direct, 2 staged, 3/4 vector loads with
  // 256/128 threads, 5/6 packed symmetric (128 threads, 85/64 registers), 7 packed
  // symmetric with the tile in shared memory by one bulk copy; 9 one warp per
  // tile, 11 the same with the block products as warp MMAs; 8 and 10, the
  // dataflow sweeps, are launched once per inner solve)
  auto launch_one = [&](int kc) {
    if (kc == 12) {
      launch_packed(P, sweep_wdf_kernel<kWdfKB>, wdf_grid, wdf_threads, wdf_smem, s, P->d_Tpdf.as<float>(),
                    P->d_tdesc.as<TileDesc>(), P->d_twin.as<int32_t>(), P->d_kddf.as<float4>(),
                    P->d_run.as<uint8_t>(), P->d_cdf.as<float2>(), P->d_dfstate.as<float4>(), npt_,
                    P->d_ctrl.as<SweepCtrl>(), P->d_partials.as<double>(), hist, hist_len, P->nparts, pp_max);
      return;
    }
    if (kc == 7) {
      auto go = [&](auto* kern, const auto* Tp) {
        launch_packed(P, kern, P->nparts, 128, symb_smem, s, Tp, P->d_tdesc.as<TileDesc>(),
                      P->d_twin.as<int32_t>(), P->d_kd32.as<float2>(), P->d_run.as<uint8_t>(),
                      P->d_c32.as<float>(), P->d_state32.as<float>(), npt_, P->d_ctrl.as<SweepCtrl>(),
                      P->d_partials.as<double>(), hist, hist_len, P->nparts, pp_max, tbuf_elems);
      };
      if (prec == VTM_PREC_FP32) go(sweep_symb_kernel<float, 128>, P->d_Tp32.as<float>());
      else with16([&](auto h) {
        using H = decltype(h);
        go(sweep_symb_kernel<H, 128>, P->d_Tp16.as<H>());
      });
      return;
    }
    if (kc == 11) {
      with16([&](auto h) {
        using H = decltype(h);
        launch_packed(P, sweep_wmma_kernel<H, kWmmaPD>, wmma_grid, wmma_threads, wmma_smem, s,
                      P->d_Tp16.as<H>(), P->d_tdesc.as<TileDesc>(), P->d_twin.as<int32_t>(),
                      P->d_kd32.as<float2>(), P->d_run.as<uint8_t>(), P->d_c32.as<float>(),
                      P->d_fstate32.as<float>(), npt_, P->d_ctrl.as<SweepCtrl>(), P->d_partials.as<double>(),
                      hist, hist_len, P->nparts, pp_max);
      });
      return;
    }
    if (kc == 9) {
      with_wsym([&](auto* kern, const auto* Tp) {
        launch_packed(P, kern, wsym_grid, wsym_threads, wsym_smem, s, Tp, P->d_tdesc.as<TileDesc>(),
                      P->d_twin.as<int32_t>(), P->d_kd32.as<float2>(), P->d_run.as<uint8_t>(),
                      P->d_c32.as<float>(), P->d_fstate32.as<float>(), npt_, P->d_ctrl.as<SweepCtrl>(),
                      P->d_partials.as<double>(), hist, hist_len, P->nparts, pp_max);
      });
      return;
    }
    if (kc == 5 || kc == 6) {
      auto go = [&](auto* kern, int nt, const auto* Tp) {
        launch_packed(P, kern, P->nparts, nt, sym_smem, s, Tp, P->d_tdesc.as<TileDesc>(),
                      P->d_twin.as<int32_t>(), P->d_kd32.as<float2>(), P->d_run.as<uint8_t>(),
                      P->d_c32.as<float>(), P->d_state32.as<float>(), npt_, P->d_ctrl.as<SweepCtrl>(),
                      P->d_partials.as<double>(), hist, hist_len, P->nparts, pp_max);
      };
      // 5: up to 85 registers (6 CTAs per SM); 6: 64 registers (8 CTAs per SM).
      // Fewer than four tiles per SM: kernel 5 with 256 threads per tile (the
      // CTAs alone cannot fill the SMs; gradient grid 1024^2 in 256 tiles:
      // 19.7 -> 13.6 us per FP32 sweep)
      const bool wide5 = kc == 5 && P->nparts < 4 * sms;
      if (prec == VTM_PREC_FP32) {
        if (wide5) go(sweep_sym_kernel<float, 256, 4, 3>, 256, P->d_Tp32.as<float>());
        else if (kc == 5) go(sweep_sym_kernel<float, 128, 4, 6>, 128, P->d_Tp32.as<float>());
        else go(sweep_sym_kernel<float, 128, 4, 8>, 128, P->d_Tp32.as<float>());
      } else {
        with16([&](auto h) {
          using H = decltype(h);
          if (wide5) go(sweep_sym_kernel<H, 256, 8, 3>, 256, P->d_Tp16.as<H>());
          else if (kc == 5) go(sweep_sym_kernel<H, 128, 8, 6>, 128, P->d_Tp16.as<H>());
          else go(sweep_sym_kernel<H, 128, 8, 8>, 128, P->d_Tp16.as<H>());
        });
      }
      return;
    }
    if (kc == 3 || kc == 4) {
      auto launch_vec = [&](auto* kern, int nt, const auto* T, const auto* c, auto* state) {
        kern<<<P->nparts, nt, vec_smem, s>>>(
            T, P->d_tdesc.as<TileDesc>(), P->d_twin.as<int32_t>(),
            kd_of<std::remove_pointer_t<decltype(state)>>(P), P->d_run.as<uint8_t>(), c, state, npt_,
            P->d_ctrl.as<SweepCtrl>(), P->d_partials.as<double>(), hist, hist_len, P->nparts, ld_max);
      };
#define VTM_VEC_LAUNCH(NT, KB)                                                                  \
  do {                                                                                          \
    if (prec == VTM_PREC_FP64)                                                                  \
      launch_vec(sweep_vec_kernel<double, double, 2, NT, KB>, NT, P->d_T64.as<double>(),        \
                 P->d_c64.as<double>(), P->d_state64.as<double>());                             \
    else if (prec == VTM_PREC_FP32)                                                             \
      launch_vec(sweep_vec_kernel<float, float, 4, NT, KB>, NT, P->d_T32.as<float>(),           \
                 P->d_c32.as<float>(), P->d_state32.as<float>());                               \
    else                                                                                        \
      with16([&](auto h) {                                                                      \
        using H = decltype(h);                                                                  \
        launch_vec(sweep_vec_kernel<H, float, 8, NT, KB>, NT, P->d_T16.as<H>(),                 \
                   P->d_c32.as<float>(), P->d_state32.as<float>());                             \
      });                                                                                       \
  } while (0)
      if (kc == 3) VTM_VEC_LAUNCH(256, 8);
      else VTM_VEC_LAUNCH(128, 4);
#undef VTM_VEC_LAUNCH
      return;
    }
    if (kc == 2) {
      if (prec == VTM_PREC_FP64)
        launch_staged(sweep_staged_kernel<double, double, 2, 4>, P->d_T64.as<double>(),
                      P->d_c64.as<double>(), P->d_state64.as<double>());
      else if (prec == VTM_PREC_FP32)
        launch_staged(sweep_staged_kernel<float, float, 4, 4>, P->d_T32.as<float>(),
                      P->d_c32.as<float>(), P->d_state32.as<float>());
      else
        with16([&](auto h) {
          using H = decltype(h);
          launch_staged(sweep_staged_kernel<H, float, 8, 4>, P->d_T16.as<H>(), P->d_c32.as<float>(),
                        P->d_state32.as<float>());
        });
      return;
    }
    if (prec == VTM_PREC_FP64)
      launch_sweep<double, double>(P, P->d_T64.as<double>(), P->d_c64.as<double>(),
                                   P->d_state64.as<double>(), threads, smem, hist, hist_len);
    else if (prec == VTM_PREC_FP32)
      launch_sweep<float, float>(P, P->d_T32.as<float>(), P->d_c32.as<float>(),
                                 P->d_state32.as<float>(), threads, smem, hist, hist_len);
    else
      with16([&](auto h) {
        using H = decltype(h);
        launch_sweep<H, float>(P, P->d_T16.as<H>(), P->d_c32.as<float>(), P->d_state32.as<float>(), threads,
                               smem, hist, hist_len);
      });
  };
  // Autotuner: on the first solve of this precision, time every kernel that
  // fits on this plan's tiles (a few sweeps each, from a zero state that is
  // reset afterwards) and keep the fastest.
  // dataflow sweeps: packed symmetric blocks, one cooperative launch per inner
  // solve, all CTAs co-resident
  int flow_grid = 0;
  if (sym_ok) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, P->device);
    const void* kfn = prec == VTM_PREC_FP32
                          ? (const void*)sweep_flow_kernel<float, 128, 4, false>
                          : pick16((const void*)sweep_flow_kernel<__nv_bfloat16, 128, 8, false>,
                                   (const void*)sweep_flow_kernel<__half, 128, 8, false>);
    int per_sm = 0;
    if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 128, sym_smem) == cudaSuccess &&
        per_sm > 0)
      flow_grid = std::min(P->nparts, per_sm * sms);
    cudaGetLastError();
  }
  const bool flow_ok = flow_grid > 0;
  // dataflow sweeps with one warp per tile: every tile resident at once
  const bool async = P->opts.method == VTM_METHOD_ASYNC;
  const void* wflow_kfn = nullptr;
  if (pp_max <= 128) {
    if (prec == VTM_PREC_FP32)
      wflow_kfn = async ? (const void*)sweep_wflow_kernel<float, kWsymKB32, true>
                        : (const void*)sweep_wflow_kernel<float, kWsymKB32, false>;
    else if (prec == VTM_PREC_BF16)
      wflow_kfn = async ? (const void*)sweep_wflow_kernel<__nv_bfloat16, kWsymKB16, true>
                        : (const void*)sweep_wflow_kernel<__nv_bfloat16, kWsymKB16, false>;
    else if (prec == VTM_PREC_FP16)
      wflow_kfn = async ? (const void*)sweep_wflow_kernel<__half, kWsymKB16, true>
                        : (const void*)sweep_wflow_kernel<__half, kWsymKB16, false>;
  }
  int wflow_grid = 0;
  if (sym_ok && wflow_kfn) {
    int coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, P->device);
    const int need = (P->nparts + kWflowWarps - 1) / kWflowWarps;
    if (coop &&
        cudaFuncSetAttribute(wflow_kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wflow_smem) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wflow_kfn, 32 * kWflowWarps, wflow_smem) ==
            cudaSuccess &&
        per_sm * sms >= need)
      wflow_grid = need;
    cudaGetLastError();
  }
  const bool wflow_ok = wflow_grid > 0;
  // counters of the dataflow kernels.  Kernel 8: 4 sweep counters, the
  // published decision at byte 32.  Kernel 10: 16 sweep counters, the
  // decision at byte 64, 16 x 32 group counters at byte 128, 16 x 32 group
  // sums at byte 2176; 16 x nparts tile partials.
  constexpr size_t kFlowBytes = 8192;
  if (flow_ok || wflow_ok) {
    VTM_TRY(dev_alloc(P->d_done, (size_t)P->nparts * sizeof(int)));
    VTM_TRY(dev_alloc(P->d_flow, kFlowBytes));
    VTM_TRY(dev_alloc(P->d_part4, 16 * (size_t)P->nparts * sizeof(double)));
  }
  // three wave slots: the dataflow kernels and the one-warp-per-tile sweeps
  if (sym_ok) VTM_TRY(dev_alloc(P->d_fstate32, 6 * (size_t)std::max<int64_t>(npt, 1) * sizeof(float)));
  // one cooperative launch runs sweeps 1.. until a flag (k_max in ctrl)
  auto launch_flow = [&]() -> cudaError_t {
    cudaMemsetAsync(P->d_done.p, 0, (size_t)P->nparts * sizeof(int), s);
    cudaMemsetAsync(P->d_flow.p, 0, kFlowBytes, s);
    const void* Tp = prec == VTM_PREC_FP32 ? P->d_Tp32.p : P->d_Tp16.p;
    const TileDesc* td = P->d_tdesc.as<TileDesc>();
    const int32_t* tw = P->d_twin.as<int32_t>();
    const float2* kdp = P->d_kd32.as<float2>();
    const uint8_t* rn = P->d_run.as<uint8_t>();
    const float* cp = P->d_c32.as<float>();
    float* st3 = P->d_fstate32.as<float>();
    const int32_t* no = P->d_nbr_off.as<int32_t>();
    const int32_t* nbp = P->d_nbr.as<int32_t>();
    int* dn = P->d_done.as<int>();
    unsigned* cnt = reinterpret_cast<unsigned*>(P->d_flow.p);
    int* gkp = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(P->d_flow.p) + 32);
    SweepCtrl* ct = P->d_ctrl.as<SweepCtrl>();
    double* p4 = P->d_part4.as<double>();
    int np = P->nparts, ppm = pp_max, hl = hist_len, k0 = 1;
    int64_t npv = npt_;
    double* hp = hist;
    uint32_t mp = (uint32_t)P->opts.wait_polls;
    int ls = P->opts.flow_lag;
    void* args[] = {&Tp, &td, &tw, &kdp, &rn, &cp, &st3, &npv, &no, &nbp, &dn, &cnt, &gkp, &ct, &p4, &hp,
                    &hl, &np, &ppm, &k0, &mp, &ls};
    const bool async = P->opts.method == VTM_METHOD_ASYNC;
    const void* kfn =
        prec == VTM_PREC_FP32
            ? (async ? (const void*)sweep_flow_kernel<float, 128, 4, true>
                     : (const void*)sweep_flow_kernel<float, 128, 4, false>)
            : (async ? pick16((const void*)sweep_flow_kernel<__nv_bfloat16, 128, 8, true>,
                              (const void*)sweep_flow_kernel<__half, 128, 8, true>)
                     : pick16((const void*)sweep_flow_kernel<__nv_bfloat16, 128, 8, false>,
                              (const void*)sweep_flow_kernel<__half, 128, 8, false>));
    return cudaLaunchCooperativeKernel(kfn, flow_grid, 128, args, sym_smem, s);
  };
  // the same with one warp per tile (kernel 10): one cooperative launch per
  // inner solve; the residual's group size G keeps at most 32 groups
  auto launch_wflow = [&]() -> cudaError_t {
    cudaMemsetAsync(P->d_done.p, 0, (size_t)P->nparts * sizeof(int), s);
    cudaMemsetAsync(P->d_flow.p, 0, kFlowBytes, s);
    const void* Tp = prec == VTM_PREC_FP32 ? P->d_Tp32.p : P->d_Tp16.p;
    const TileDesc* td = P->d_tdesc.as<TileDesc>();
    const int32_t* tw = P->d_twin.as<int32_t>();
    const float2* kdp = P->d_kd32.as<float2>();
    const uint8_t* rn = P->d_run.as<uint8_t>();
    const float* cp = P->d_c32.as<float>();
    float* st3 = P->d_fstate32.as<float>();
    const int32_t* no = P->d_nbr_off.as<int32_t>();
    const int32_t* nbp = P->d_nbr.as<int32_t>();
    int* dn = P->d_done.as<int>();
    unsigned char* fb = reinterpret_cast<unsigned char*>(P->d_flow.p);
    unsigned* cnt = reinterpret_cast<unsigned*>(fb);
    int* gkp = reinterpret_cast<int*>(fb + 64);
    unsigned* gcnt = reinterpret_cast<unsigned*>(fb + 128);
    double* gs = reinterpret_cast<double*>(fb + 2176);
    int G = std::max(1, (P->nparts + 31) / 32);
    SweepCtrl* ct = P->d_ctrl.as<SweepCtrl>();
    double* p4 = P->d_part4.as<double>();
    int np = P->nparts, ppm = pp_max, hl = hist_len, k0 = 1;
    int64_t npv = npt_;
    double* hp = hist;
    uint32_t mp = (uint32_t)P->opts.wait_polls;
    int ls = P->opts.flow_lag;
    void* args[] = {&Tp, &td, &tw, &kdp, &rn, &cp, &st3, &npv, &no, &nbp, &dn, &cnt, &gkp, &gcnt, &gs, &G,
                    &ct, &p4, &hp, &hl, &np, &ppm, &k0, &mp, &ls};
    return cudaLaunchCooperativeKernel(wflow_kfn, wflow_grid, 32 * kWflowWarps, args, wflow_smem, s);
  };
  const bool symload = ((choice == 5 || choice == 6 || choice == 9) && sym_ok) || (choice == 7 && symb_ok) ||
                       (choice == 8 && flow_ok) || (choice == 10 && wflow_ok) || (choice == 11 && wmma_ok) ||
                       (choice == 12 && wdf_ok);
  if (P->opts.method == VTM_METHOD_ASYNC && !flow_ok && !wflow_ok) {
    set_detail("vtm_solve: asynchronous VTM runs on the packed symmetric dataflow kernel: it needs "
               "FP32/BF16/FP16 sweeps of a symmetric plan with at most 256 ports per sub-circuit");
    return VTM_EINVAL;
  }
  if (sym_ok) {
    cudaError_t e = cudaSuccess;
    with_wsym([&](auto* kern, const auto*) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsym_smem);
    });
    VTM_CUDA_TRY(e);
  }
  if (wmma_ok) {
    VTM_CUDA_TRY(cudaFuncSetAttribute(pick16((const void*)sweep_wmma_kernel<__nv_bfloat16, kWmmaPD>,
                                             (const void*)sweep_wmma_kernel<__half, kWmmaPD>),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wmma_smem));
  }
  if (symb_ok) {
    VTM_CUDA_TRY(cudaFuncSetAttribute(prec == VTM_PREC_FP32
                                          ? (const void*)sweep_symb_kernel<float, 128>
                                          : pick16((const void*)sweep_symb_kernel<__nv_bfloat16, 128>,
                                                   (const void*)sweep_symb_kernel<__half, 128>),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)symb_smem));
  }

  int kern = (vecload || symload) ? choice : (staged ? 2 : 1);
  if (P->opts.method == VTM_METHOD_ASYNC) kern = wflow_ok ? 10 : 8;  // its own iteration: not autotuned
  else if (P->opts.sweep_kernel == 0) {
    if (P->tuned_kernel[prec] == 0) {
      const bool can_st = nv_max <= 4 * 256 && st_smem <= 200 * 1024;
      const bool can_vec = nv_max <= 256;
      const bool can_vec128 = nv_max <= 128;
      float best = 1e30f;
      int best_k = 1;
      for (int cand = 1; cand <= 12; ++cand) {
        if ((cand == 2 && !can_st) || (cand == 3 && !can_vec) || (cand == 4 && !can_vec128) ||
            ((cand == 5 || cand == 6 || cand == 9) && !sym_ok) || (cand == 7 && !symb_ok) ||
            (cand == 8 && !flow_ok) || (cand == 10 && !wflow_ok) || (cand == 11 && !wmma_ok) ||
            (cand == 12 && !wdf_ok))
          continue;
        if (cand == 8 || cand == 10) {  // one launch of 8 sweeps, per-sweep time against the others' 6
          SweepCtrl t = h;
          t.k_max = 8;
          t.tol2 = -1.0;
          t.stall = 0;
          *P->h_ctrl = t;
          VTM_TRY(upload_ctrl(P, s));
          VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
          VTM_CUDA_TRY(cand == 10 ? launch_wflow() : launch_flow());
          VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
          VTM_CUDA_TRY(cudaEventSynchronize(P->evs1));
          float ms = 0.f;
          VTM_CUDA_TRY(cudaEventElapsedTime(&ms, P->evs0, P->evs1));
          P->launch_count += 1;
          VTM_CUDA_TRY(cudaMemcpy(P->h_ctrl, P->d_ctrl.p, sizeof(SweepCtrl), cudaMemcpyDeviceToHost));
          if (P->h_ctrl->flag == 5) {
            set_detail("vtm_solve: a bounded wait of the dataflow sweeps ran out");
            return VTM_ETIMEOUT;
          }
          if (ms * 6.0f / 8.0f < best) {
            best = ms * 6.0f / 8.0f;
            best_k = cand;
          }
          continue;
        }
        if (cand == 2)
          VTM_CUDA_TRY(
              cudaFuncSetAttribute(staged_kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st_smem));
        SweepCtrl t = h;
        t.k_max = 1 << 30;
        t.tol2 = -1.0;  // never converges while timing
        t.stall = 0;
        *P->h_ctrl = t;
        VTM_TRY(upload_ctrl(P, s));
        for (int i = 0; i < 2; ++i) launch_one(cand);
        VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
        for (int i = 0; i < 6; ++i) launch_one(cand);
        VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
        VTM_CUDA_TRY(cudaGetLastError());
        VTM_CUDA_TRY(cudaEventSynchronize(P->evs1));
        float ms = 0.f;
        VTM_CUDA_TRY(cudaEventElapsedTime(&ms, P->evs0, P->evs1));
        P->launch_count += 8;
        if (ms < best) {
          best = ms;
          best_k = cand;
        }
      }
      P->tuned_kernel[prec] = best_k;
      P->tuned_ms[prec] = best / 6.0f;
      // back to the initial state of this inner solve
      *P->h_ctrl = h;
      VTM_TRY(upload_ctrl(P, s));
      if (prec == VTM_PREC_FP64)
        VTM_CUDA_TRY(cudaMemsetAsync(P->d_state64.p, 0, 4 * npt * sizeof(double), s));
      else
        VTM_CUDA_TRY(cudaMemsetAsync(P->d_state32.p, 0, 4 * npt * sizeof(float), s));
    }
    kern = P->tuned_kernel[prec];
    if (kern == 2)
      VTM_CUDA_TRY(cudaFuncSetAttribute(staged_kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st_smem));
  }
  if (kern == 2 && !st_grid) {  // occupancy query before any capture
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, staged_kfn, st_threads, st_smem);
    st_grid = std::max(1, std::min(P->nparts, std::max(per_sm, 1) * sms));
  }
  P->dataflow_kernel = kern;
  if (kern == 8 || kern == 10) {
    VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
    VTM_CUDA_TRY(kern == 10 ? launch_wflow() : launch_flow());
    VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
    VTM_CUDA_TRY(cudaMemcpyAsync(P->h_ctrl, P->d_ctrl.p, sizeof(SweepCtrl), cudaMemcpyDeviceToHost, s));
    VTM_CUDA_TRY(cudaStreamSynchronize(s));
    float bms = 0.f;
    VTM_CUDA_TRY(cudaEventElapsedTime(&bms, P->evs0, P->evs1));
    P->sweep_ms += bms;
    const SweepCtrl& r = *P->h_ctrl;
    P->sweep_launch_count += std::max(r.k - 1, 1);  // sweeps run by the one launch
    P->launch_count += 1;
    if (r.flag == 5) {
      set_detail("vtm_solve: a bounded wait of the dataflow sweeps ran out");
      return VTM_ETIMEOUT;
    }
    *flag_out = r.flag;
    *sweep_out = (r.flag == 1 || r.flag == 4) ? r.conv_sweep : std::min(r.k - 1, budget);
    P->wave_slot = P->d_fstate32.as<float>() +
                   (P->opts.method == VTM_METHOD_ASYNC ? 0 : (size_t)(*sweep_out % 3) * npt * 2);
    return VTM_OK;
  }
  // Batches of check_every launches, captured once into a CUDA graph when the
  // plan has its own stream (launches past convergence or the sweep limit
  // return at once, so full batches are always safe), and a graph of a
  // quarter batch for the tail up to a hinted count.
  const int batch = P->opts.check_every;
  const int sbatch = std::max(1, batch / 4);
  cudaGraphExec_t gexec = nullptr, gsmall = nullptr;
  if (P->stream && P->opts.graphs != 1) {
    SweepGraph& G = P->sweep_graph[prec];
    const uint64_t key = ((uint64_t)kern << 56) ^ ((uint64_t)(P->opts.pdl == 1) << 52) ^
                         ((uint64_t)batch << 32) ^ (uint64_t)(uintptr_t)hist ^ ((uint64_t)hist_len << 16);
    if (!G.exec || G.key != key) {
      G.reset();
      for (int g = 0; g < 2; ++g) {
        cudaGraph_t graph = nullptr;
        VTM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < (g ? sbatch : batch); ++i) launch_one(kern);
        VTM_CUDA_TRY(cudaStreamEndCapture(s, &graph));
        cudaGraphExec_t& ex = g ? G.small : G.exec;
        cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          ex = nullptr;
          cudaGetLastError();
        }
      }
      if (G.exec) G.key = key;
    }
    gexec = G.exec;
    gsmall = G.small;
  }
  // hint: the sweeps the same refinement step took last time.  The launches
  // up to the one that decides that sweep (launch k decides sweep k - 1; the
  // dataflow kernels decide one launch later), as whole batches and then
  // quarter batches, go out before the first poll of the flag: a poll costs a
  // host round trip with the GPU idle, a launch that finds the solve
  // converged returns at once.
  int launched = 0;
  int reps = 1, sreps = 0;
  const int lag = (kern == 9 || kern == 11) ? 2 : 1;  // launches past the hinted sweep
  const int need = hint > 0 ? std::min(hint + lag, budget + lag) : 0;
  if (gexec && need > 0) {
    reps = std::min(need / batch, 64);
    sreps = gsmall ? (need - reps * batch + sbatch - 1) / sbatch : 0;
    if (!gsmall && reps * batch < need) ++reps;
    if (reps + sreps == 0) reps = 1;
  }
  // without graphs the first round is the hinted count of single launches
  int first = need;
  while (true) {
    const int m = gexec ? batch : std::min(first > 0 ? first : batch, budget + 1 - launched);
    first = 0;
    VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
    if (gexec) {
      for (int i = 0; i < reps; ++i) VTM_CUDA_TRY(cudaGraphLaunch(gexec, s));
      for (int i = 0; i < sreps; ++i) VTM_CUDA_TRY(cudaGraphLaunch(gsmall, s));
    } else {
      for (int i = 0; i < m; ++i) launch_one(kern);
    }
    const int went = gexec ? reps * batch + sreps * sbatch : m;
    launched += went;
    VTM_CUDA_TRY(cudaGetLastError());
    VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
    VTM_CUDA_TRY(cudaMemcpyAsync(P->h_ctrl, P->d_ctrl.p, sizeof(SweepCtrl), cudaMemcpyDeviceToHost, s));
    VTM_CUDA_TRY(cudaStreamSynchronize(s));
    float bms = 0.f;
    VTM_CUDA_TRY(cudaEventElapsedTime(&bms, P->evs0, P->evs1));
    P->sweep_ms += bms;
    P->sweep_launch_count += went;
    P->launch_count += went;
    reps = 1;
    sreps = 0;
    if (P->h_ctrl->flag || launched > budget) break;
  }
  const SweepCtrl& r = *P->h_ctrl;
  if (r.flag == 5) {
    set_detail("vtm_solve: a bounded wait for a bulk copy ran out");
    return VTM_ETIMEOUT;
  }
  *flag_out = r.flag;
  if (r.flag == 1 || r.flag == 4) *sweep_out = r.conv_sweep;
  else *sweep_out = std::min(r.k - 1, budget);
  if (kern == 12) {
    // the chosen double-float slot as FP64 pairs for the recovery
    join_df_kernel<<<grid_for(std::max<int64_t>(npt, 1)), 256, 0, s>>>(
        P->d_dfstate.as<float4>() + (size_t)(*sweep_out % 3) * npt, P->d_state64.as<double>(), npt);
    VTM_CUDA_TRY(cudaGetLastError());
    P->launch_count++;
    P->wave_slot = P->d_state64.as<double>();
  } else if (prec == VTM_PREC_FP64)
    P->wave_slot = P->d_state64.as<double>() + (size_t)(*sweep_out & 1) * npt * 2;
  else if (kern == 9 || kern == 11)  // three slots
    P->wave_slot = P->d_fstate32.as<float>() + (size_t)(*sweep_out % 3) * npt * 2;
  else
    P->wave_slot = P->d_state32.as<float>() + (size_t)(*sweep_out & 1) * npt * 2;
  return VTM_OK;
}

static vtm_status norms(vtm_plan_s* P, const double* x, const double* b, double* r, double* rr,
                        double* bb, float* v1 = nullptr, float* v2 = nullptr) {
  return residual_pair(P, x, b, r, rr, bb, v1, v2);
}

// The ELL copy of A for the single-column residual, built on first use after
// each set of values when every row has at most 8 entries and the padding
// stays under half of the nonzeros (else the CSR kernel serves)
static vtm_status ensure_ell(vtm_plan_s* P) {
  if (P->ell_state != 0) return VTM_OK;
  int64_t maxlen = 0;
  for (int64_t i = 0; i < P->n; ++i) maxlen = std::max(maxlen, P->h_rowptr[i + 1] - P->h_rowptr[i]);
  if (maxlen < 1 || maxlen > 8 || P->n * maxlen > P->nnz + P->nnz / 2) {
    P->ell_state = 2;
    return VTM_OK;
  }
  P->ell_k = (int)maxlen;
  VTM_TRY(dev_alloc(P->d_ell_val, (size_t)P->n * maxlen * sizeof(double)));
  VTM_TRY(dev_alloc(P->d_ell_col, (size_t)P->n * maxlen * sizeof(int32_t)));
  ell_build_kernel<<<grid_for(P->n), 256, 0, P->stream>>>(P->d_rowptr.as<int64_t>(), P->d_colidx.as<int32_t>(),
                                                           P->d_vals.as<double>(), P->n, P->ell_k,
                                                           P->d_ell_val.as<double>(), P->d_ell_col.as<int32_t>());
  VTM_CUDA_TRY(cudaGetLastError());
  P->launch_count++;
  P->ell_state = 1;
  return VTM_OK;
}

vtm_status residual_pair(vtm_plan_s* P, const double* x, const double* b, double* r, double* rr,
                         double* bb, float* v1, float* v2) {
  cudaStream_t s = P->stream;
  const int grid = grid_for(P->n);
  double* out = P->d_red.as<double>() + 2;
  unsigned* counter = reinterpret_cast<unsigned*>(P->d_red.p);
  VTM_TRY(ensure_ell(P));
  if (v1 && P->ell_state != 1) return VTM_EINTERNAL;  // callers ask for v1 only with the ELL copy
  if (v1 && !P->d_iperm.p) VTM_TRY(upload(P->d_iperm, P->iperm, s));
  P->launch_count++;
  if (P->ell_state == 1) {
    auto go = [&](auto kern) {
      kern<<<grid, 256, 0, s>>>(P->d_ell_val.as<double>(), P->d_ell_col.as<int32_t>(), x, b, r, P->n,
                                P->d_iperm.as<int32_t>(), v1, v2, P->d_partials.as<double>(), counter, out);
    };
    switch (P->ell_k) {
      case 1: go(residual_ell_kernel<1>); break;
      case 2: go(residual_ell_kernel<2>); break;
      case 3: go(residual_ell_kernel<3>); break;
      case 4: go(residual_ell_kernel<4>); break;
      case 5: go(residual_ell_kernel<5>); break;
      case 6: go(residual_ell_kernel<6>); break;
      case 7: go(residual_ell_kernel<7>); break;
      default: go(residual_ell_kernel<8>); break;
    }
  } else {
    residual_kernel<<<grid, 256, 0, s>>>(P->d_rowptr.as<int64_t>(), P->d_colidx.as<int32_t>(),
                                         P->d_vals.as<double>(), x, b, r, P->n,
                                         P->d_partials.as<double>(), counter, out);
  }
  VTM_CUDA_TRY(cudaGetLastError());
  double h[2];
  VTM_CUDA_TRY(cudaMemcpyAsync(h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  *rr = h[0];
  *bb = h[1];
  return VTM_OK;
}

// Solve one column: d_b (global order) -> d_x (global order).
// One right-hand side.  d_x0 (device, may be NULL): warm start -- the
// refinement starts from x = d_x0 (its first inner problem is A d = b - A x0).
static vtm_status solve_one(vtm_plan_s* P, const double* d_b, double* d_x, double tol,
                            vtm_info* info, bool record_hist, const double* d_x0 = nullptr) {
  cudaStream_t s = P->stream;
  const int64_t n = P->n;
  const int64_t npt = (int64_t)P->port_node.size();
  const int prec = P->opts.precision;
  const int g1 = grid_for(n), g2 = grid_for(std::max<int64_t>(npt, 1));
  double* v = P->d_v.as<double>();
  double* xacc = P->d_xacc.as<double>();
  double* r = P->d_r.as<double>();
  if (prec != VTM_PREC_FP64) {
    VTM_TRY(dev_alloc(P->d_c32, std::max<int64_t>(npt, 1) * sizeof(float)));
    VTM_TRY(dev_alloc(P->d_state32, 4 * std::max<int64_t>(npt, 1) * sizeof(float)));
  }
  double rr0, bb;
  // BF16/FP16 steps run both band solves in FP32; with the ELL residual the
  // residual kernel writes their right-hand sides (r rounded to FP32, band
  // order) itself: v32 for the first solve, v32b for the recovery
  VTM_TRY(ensure_ell(P));
  const bool fuse = (prec == VTM_PREC_BF16 || prec == VTM_PREC_FP16) && !P->general && npt > 0 &&
                    P->d_Lc32.p && P->ell_state == 1;
  float* v32 = nullptr;
  float* v32b = nullptr;
  if (fuse) {
    VTM_TRY(dev_alloc(P->d_v32, (size_t)n * sizeof(float)));
    VTM_TRY(dev_alloc(P->d_v32b, (size_t)n * sizeof(float)));
    v32 = P->d_v32.as<float>();
    v32b = P->d_v32b.as<float>();
  }
  // ||b||^2 and r = b - A x (x = 0 gives r = b)
  const bool warm = d_x0 != nullptr;
  if (warm)
    VTM_CUDA_TRY(cudaMemcpyAsync(xacc, d_x0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    VTM_CUDA_TRY(cudaMemsetAsync(xacc, 0, n * sizeof(double), s));
  VTM_TRY(norms(P, xacc, d_b, fuse ? nullptr : r, &rr0, &bb, v32, v32b));
  const double bnorm = std::sqrt(bb);
  info->sweeps = 0;
  info->outer_steps = 0;
  info->relres = 0.0;
  info->first_sweep_converged = 0;
  if (bb == 0.0) {
    VTM_CUDA_TRY(cudaMemsetAsync(d_x, 0, n * sizeof(double), s));
    return VTM_OK;
  }
  const double target = tol * bnorm;
  double rnorm = warm ? std::sqrt(rr0) : bnorm;
  if (warm && rnorm <= target) {  // the start already meets the tolerance
    info->relres = rnorm / bnorm;
    VTM_CUDA_TRY(cudaMemcpyAsync(d_x, xacc, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    VTM_CUDA_TRY(cudaStreamSynchronize(s));
    return VTM_OK;
  }
  // Default inner tolerance: FP32 sweeps gain five digits per refinement step
  // (two steps reach 1e-10), BF16 sweeps two and a half (measured: 3e-3 takes
  // one step less than 1e-2 on the power grid and the thermal grid).
  double inner_tol = P->opts.inner_tol;
  if (inner_tol <= 0) inner_tol = default_inner_tol(prec);
  const int max_outer = (prec == VTM_PREC_FP64 || P->general) ? 4 : P->opts.max_outer;
  int sweeps_left = P->opts.max_sweeps;
  vtm_status result = VTM_ENOCONV;
  bool stalled = false;
  for (int outer = 0; outer < max_outer; ++outer) {
    // inner problem A d = r (r = b at the first step of a cold start)
    const double* rhs = (outer == 0 && !warm) ? d_b : r;
    const int accumulate = (outer > 0 || warm) ? 1 : 0;
    // x0 = K_P^-1 rhs_P: FP64, or FP32 for a low-precision inner solve (it
    // only feeds c, whose error the next refinement step removes)
    const bool x0_f32 = prec != VTM_PREC_FP64 && !P->general && npt > 0 && P->d_Lc32.p;
    if (x0_f32) {
      VTM_TRY(dev_alloc(P->d_v32, (size_t)n * sizeof(float)));
      if (!fuse) {
        gather_perm_f32_kernel<<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, P->d_v32.as<float>(), n);
        P->launch_count++;
      }
      launch_band_solve32(P, P->d_v32.as<float>(), 1, n, s);
    } else {
      gather_perm_kernel<<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, v, n);
      P->launch_count++;
      launch_band_solve(P, v, 1, n, s);
    }
    int kc = 0, flag = 1;
    bool recovered_f32 = false;
    if (P->general && P->n_in > 0) {
      // channel form (lagged couplings / block Jacobi), FP64 sweeps
      VTM_TRY(general_const(P, v));
      double* hist = (record_hist && outer == 0 && P->opts.history) ? P->d_hist.as<double>() : nullptr;
      const int hist_len = hist ? P->opts.history_len : 0;
      if (hist) VTM_CUDA_TRY(cudaMemsetAsync(hist, 0, hist_len * sizeof(double), s));
      if (sweeps_left <= 0) break;
      VTM_TRY(general_sweeps(P, rnorm * rnorm, target * target, sweeps_left, hist, hist_len, &kc, &flag));
      if (hist)
        VTM_CUDA_TRY(cudaMemcpyAsync(P->opts.history, hist, hist_len * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
      if (outer == 0 && flag == 1) info->first_sweep_converged = kc;
      info->sweeps += kc;
      sweeps_left -= kc;
      gather_perm_kernel<<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, v, n);
      P->launch_count++;
      VTM_TRY(general_inject(P, kc, v));
      launch_band_solve(P, v, 1, n, s);
    } else if (!P->general && npt > 0) {
      if (prec == VTM_PREC_FP64)
        port_const_kernel<double, double><<<g2, 256, 0, s>>>(
            P->d_port_pos.as<int32_t>(), P->d_bout.as<double>(), v, P->d_c64.as<double>(), npt);
      else if (x0_f32)
        port_const_kernel<float, float><<<g2, 256, 0, s>>>(P->d_port_pos.as<int32_t>(),
                                                           P->d_bout.as<double>(), P->d_v32.as<float>(),
                                                           P->d_c32.as<float>(), npt);
      else
        port_const_kernel<float, double><<<g2, 256, 0, s>>>(
            P->d_port_pos.as<int32_t>(), P->d_bout.as<double>(), v, P->d_c32.as<float>(), npt);
      VTM_CUDA_TRY(cudaGetLastError());
      P->launch_count++;
      // a low-precision inner solve that can finish the job aims below the
      // target (the rounding of its waves and of c is on top); earlier ones
      // stop at inner_tol
      double t_abs = target;
      if (prec != VTM_PREC_FP64)
        t_abs = inner_tol * rnorm <= 4.0 * target ? 0.5 * target : std::max(target, inner_tol * rnorm);
      double* hist = (record_hist && outer == 0 && P->opts.history) ? P->d_hist.as<double>() : nullptr;
      const int hist_len = hist ? P->opts.history_len : 0;
      if (hist) VTM_CUDA_TRY(cudaMemsetAsync(hist, 0, hist_len * sizeof(double), s));
      if (sweeps_left <= 0) break;
      // low-precision inner solves stop at their rounding floor as well
      const int stall = prec == VTM_PREC_FP64 ? 0 : 64;
      const int step = std::min(outer, 7);
      VTM_TRY(run_sweeps(P, rnorm * rnorm, t_abs * t_abs, sweeps_left, prec, hist, hist_len, stall,
                         &kc, &flag, P->sweep_hint[prec][step]));
      P->sweep_hint[prec][step] = kc;
      if (hist) {
        VTM_CUDA_TRY(cudaMemcpyAsync(P->opts.history, hist, hist_len * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
      }
      if (outer == 0 && flag == 1) info->first_sweep_converged = kc;
      info->sweeps += kc;
      sweeps_left -= kc;
      // recovery of the sweep kc: x_P = K_P^-1 (rhs_P + B beta w_in).  An
      // FP32 recovery leaves ~1e-7 cond(K_P) relative error in the correction
      // (6e-5 on the power grid): below what a BF16 step gains (1e-2), so BF16
      // steps recover in FP32; FP32 steps gain five digits and recover in FP64.
      P->launch_count += 2;
      const float* slot32 = static_cast<const float*>(P->wave_slot);
      recovered_f32 = (prec == VTM_PREC_BF16 || prec == VTM_PREC_FP16) && x0_f32;
      if (recovered_f32) {
        float* vr = fuse ? v32b : P->d_v32.as<float>();
        if (!fuse) gather_perm_f32_kernel<<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, vr, n);
        inject_kernel<float, float><<<g2, 256, 0, s>>>(P->d_port_pos.as<int32_t>(), P->d_run.as<uint8_t>(),
                                                      P->d_beta.as<double>(), slot32, vr, npt);
        launch_band_solve32(P, vr, 1, n, s);
      } else {
        gather_perm_kernel<<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), rhs, v, n);
        if (prec == VTM_PREC_FP64)
          inject_kernel<double, double><<<g2, 256, 0, s>>>(
              P->d_port_pos.as<int32_t>(), P->d_run.as<uint8_t>(), P->d_beta.as<double>(),
              static_cast<const double*>(P->wave_slot), v, npt);
        else
          inject_kernel<float, double><<<g2, 256, 0, s>>>(P->d_port_pos.as<int32_t>(), P->d_run.as<uint8_t>(),
                                                         P->d_beta.as<double>(), slot32, v, npt);
        launch_band_solve(P, v, 1, n, s);
      }
    } else {
      info->sweeps += 1;  // one direct solve per sub-circuit
      if (outer == 0) info->first_sweep_converged = 1;
    }
    if (recovered_f32)
      scatter_perm_kernel<float><<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), fuse ? v32b : P->d_v32.as<float>(),
                                                    xacc, n, accumulate);
    else
      scatter_perm_kernel<double><<<g1, 256, 0, s>>>(P->d_perm.as<int32_t>(), v, xacc, n, accumulate);
    P->launch_count++;
    VTM_CUDA_TRY(cudaGetLastError());
    info->outer_steps = outer + 1;
    double rr;
    VTM_TRY(norms(P, xacc, d_b, fuse ? nullptr : r, &rr, &bb, v32, v32b));
    const double rprev = rnorm;
    rnorm = std::sqrt(rr);
    info->relres = rnorm / bnorm;
    if (flag == 3 || !std::isfinite(rnorm)) {
      result = VTM_EDIVERGED;
      break;
    }
    if (rnorm <= target) {
      result = VTM_OK;
      break;
    }
    if (flag == 2 || sweeps_left <= 0) {
      result = VTM_ENOCONV;
      break;
    }
    if (!P->general && refinement_stalled(prec, rprev, rnorm, target)) {
      result = VTM_ENOCONV;
      stalled = true;
      break;
    }
  }
  VTM_CUDA_TRY(cudaMemcpyAsync(d_x, xacc, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  if (result == VTM_ENOCONV)
    set_detail(stalled ? "vtm_solve: refinement stalled (step " + std::to_string(info->outer_steps) +
                             " cut ||r|| by less than " + std::to_string((int)refinement_min_gain(prec)) + "x)"
                       : std::string("vtm_solve: tolerance not met"));
  if (result == VTM_EDIVERGED) set_detail("vtm_solve: the iteration diverged");
  return result;
}

vtm_status solve_columns(vtm_plan_s* P, const double* d_b, double* d_x, int64_t nrhs, double tol,
                         vtm_info* info) {
  // several right-hand sides: one batched iteration (up to 64 per pass)
  const bool batch = P->opts.batch != 1 && nrhs >= 2 && !P->general && !P->port_node.empty() &&
                     P->opts.method != VTM_METHOD_ASYNC;  // asynchronous VTM: column by column
  if (batch) {
    vtm_status worst = VTM_OK;
    vtm_info agg{};
    for (int64_t c0 = 0; c0 < nrhs; c0 += 64) {
      const int R = (int)std::min<int64_t>(64, nrhs - c0);
      vtm_info one{};
      vtm_status st = solve_batched(P, d_b + c0 * P->n, d_x + c0 * P->n, R, tol, &one, c0 == 0);
      if (st != VTM_OK && st != VTM_ENOCONV && st != VTM_EDIVERGED) return st;
      if (st != VTM_OK && worst == VTM_OK) worst = st;
      agg.sweeps = std::max(agg.sweeps, one.sweeps);
      agg.outer_steps = std::max(agg.outer_steps, one.outer_steps);
      agg.relres = std::max(agg.relres, one.relres);
      if (c0 == 0) agg.first_sweep_converged = one.first_sweep_converged;
    }
    *info = agg;
    return worst;
  }
  vtm_info agg{};
  vtm_status worst = VTM_OK;
  for (int64_t col = 0; col < nrhs; ++col) {
    vtm_info one{};
    vtm_status st = solve_one(P, d_b + col * P->n, d_x + col * P->n, tol, &one, col == 0);
    if (st != VTM_OK && st != VTM_ENOCONV && st != VTM_EDIVERGED) return st;
    if (st != VTM_OK && worst == VTM_OK) worst = st;
    agg.sweeps = std::max(agg.sweeps, one.sweeps);
    agg.outer_steps = std::max(agg.outer_steps, one.outer_steps);
    agg.relres = std::max(agg.relres, one.relres);
    if (col == 0) agg.first_sweep_converged = one.first_sweep_converged;
  }
  *info = agg;
  return worst;
}

vtm_status residual_norms(vtm_plan_s* P, const double* d_x, const double* d_b, int64_t nrhs,
                          double* rel) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double rr, bb;
    VTM_TRY(norms(P, d_x + c * P->n, d_b + c * P->n, nullptr, &rr, &bb));
    rel[c] = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
  }
  return VTM_OK;
}

}  // namespace vtm

using namespace vtm;

// Host/device staging of the caller's vectors.
// A host array seen by the device: host input arrays are copied into, and
// host outputs computed in, device buffers the plan keeps (slot 0..2; grown
// when a call needs more), so repeated calls with host buffers allocate
// nothing (an allocation and its release would synchronise the device).
struct Staged {
  const double* in_dev = nullptr;
  double* out_dev = nullptr;
  bool out_host = false;
};

static vtm_status stage(vtm_plan_s* P, const double* in, double* out, int64_t count, Staged& S, int slot = 0) {
  if (is_device_ptr(in)) {
    S.in_dev = in;
  } else {
    DevBuf& t = P->d_stage_in[slot];
    VTM_TRY(dev_alloc(t, count * sizeof(double)));
    VTM_CUDA_TRY(cudaMemcpyAsync(t.p, in, count * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    S.in_dev = t.as<double>();
  }
  if (out) {
    if (is_device_ptr(out)) {
      S.out_dev = out;
    } else {
      DevBuf& t = P->d_stage_out[slot];
      VTM_TRY(dev_alloc(t, count * sizeof(double)));
      S.out_dev = t.as<double>();
      S.out_host = true;
    }
  }
  return VTM_OK;
}

static vtm_status solve_entry(vtm_plan_s* P, const double* b, double* x, int64_t nrhs, double tol,
                              vtm_info* info) {
  if (!P || !b || !x || nrhs <= 0 || !(tol > 0)) return VTM_EINVAL;
  if (!P->factored) return VTM_ENOTFACTORED;
  cudaSetDevice(P->device);
  vtm_info local{};
  if (!info) info = &local;
  Staged S;
  const int64_t count = P->n * nrhs;
  VTM_TRY(stage(P, b, x, count, S));
  P->launch_count = 0;
  P->sweep_launch_count = 0;
  P->sweep_ms = 0.0;
  VTM_CUDA_TRY(cudaEventRecord(P->ev0, P->stream));
  vtm_status st = solve_columns(P, S.in_dev, S.out_dev, nrhs, tol, info);
  VTM_CUDA_TRY(cudaEventRecord(P->ev1, P->stream));
  if (S.out_host)
    VTM_CUDA_TRY(cudaMemcpyAsync(x, S.out_dev, count * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  VTM_CUDA_TRY(cudaStreamSynchronize(P->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, P->ev0, P->ev1);
  info->t_solve_ms = ms;
  info->kernel_launches = P->launch_count;
  info->sweep_launches = P->sweep_launch_count;
  info->t_sweeps_ms = P->sweep_ms;
  return st;
}

extern "C" vtm_status vtm_solve(vtm_plan_t P, const double* b, double* x, int64_t nrhs, double tol,
                                vtm_info* info) {
  return solve_entry(P, b, x, nrhs, tol, info);
}

// b_k = p_k + cdiag .* x_{k-1}  (x_{k-1} = NULL: zero initial state)
__global__ void march_rhs_kernel(const double* __restrict__ p, const double* __restrict__ cdiag,
                                 const double* __restrict__ xprev, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = xprev ? p[i] + cdiag[i] * xprev[i] : p[i];
}

extern "C" vtm_status vtm_march(vtm_plan_t P, const double* cdiag, const double* p, const double* x0,
                                double* X, int64_t nsteps, double tol, vtm_info* info) {
  if (!P || !cdiag || !p || !X || nsteps <= 0 || !(tol > 0)) return VTM_EINVAL;
  if (!P->factored) return VTM_ENOTFACTORED;
  cudaSetDevice(P->device);
  vtm_info local{};
  if (!info) info = &local;
  *info = vtm_info{};
  const int64_t n = P->n;
  Staged Sp, Sc, S0;
  VTM_TRY(stage(P, p, X, n * nsteps, Sp, 0));
  VTM_TRY(stage(P, cdiag, nullptr, n, Sc, 1));
  if (x0) VTM_TRY(stage(P, x0, nullptr, n, S0, 2));
  DevBuf bk;
  VTM_TRY(dev_alloc(bk, (size_t)n * sizeof(double)));
  P->launch_count = 0;
  P->sweep_launch_count = 0;
  P->sweep_ms = 0.0;
  VTM_CUDA_TRY(cudaEventRecord(P->ev0, P->stream));
  vtm_status st = VTM_OK;
  for (int64_t k = 0; k < nsteps; ++k) {
    const double* xprev = k == 0 ? (x0 ? S0.in_dev : nullptr) : Sp.out_dev + (k - 1) * n;
    march_rhs_kernel<<<grid_for(n), 256, 0, P->stream>>>(Sp.in_dev + k * n, Sc.in_dev, xprev,
                                                          bk.as<double>(), n);
    P->launch_count++;
    vtm_info one{};
    // each step starts from the previous state (warm start)
    st = solve_one(P, bk.as<double>(), Sp.out_dev + k * n, tol, &one, k == 0, xprev);
    info->sweeps += one.sweeps;
    info->outer_steps += one.outer_steps;
    info->relres = std::max(info->relres, one.relres);
    if (k == 0) info->first_sweep_converged = one.first_sweep_converged;
    if (st != VTM_OK) {
      set_detail("vtm_march: step " + std::to_string(k) + ": " + vtm_strerror(st));
      break;
    }
  }
  VTM_CUDA_TRY(cudaEventRecord(P->ev1, P->stream));
  if (Sp.out_host)
    VTM_CUDA_TRY(cudaMemcpyAsync(X, Sp.out_dev, n * nsteps * sizeof(double), cudaMemcpyDeviceToHost,
                                 P->stream));
  VTM_CUDA_TRY(cudaStreamSynchronize(P->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, P->ev0, P->ev1);
  info->t_solve_ms = ms;
  info->kernel_launches = P->launch_count;
  info->sweep_launches = P->sweep_launch_count;
  info->t_sweeps_ms = P->sweep_ms;
  return st;
}

extern "C" vtm_status vtm_adjoint(vtm_plan_t P, const double* g, double* lam, int64_t nrhs,
                                  double tol, vtm_info* info) {
  if (!P) return VTM_EINVAL;
  if (P->symmetric) return solve_entry(P, g, lam, nrhs, tol, info);
  if (!P->factored) return VTM_ENOTFACTORED;
  if (!P->transposed) {
    // A^T in CSR = A in CSC
    const int64_t n = P->n;
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> ci(P->nnz);
    std::vector<double> va(P->nnz);
    for (int64_t q = 0; q < P->nnz; ++q) rp[P->h_colidx[q] + 1]++;
    for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
        int64_t d = fill[P->h_colidx[q]]++;
        ci[d] = (int32_t)i;
        va[d] = P->h_vals[q];
      }
    vtm_plan_t T = nullptr;
    VTM_TRY(vtm_plan(n, rp.data(), ci.data(), va.data(), P->h_part.data(), P->nparts, P->Zc, &P->opts,
                     P->stream, &T));
    // the same lines (the tearing is symmetric in i, j) with the same admittances
    vtm_status st = P->w_kind == VTM_W_ALPHA
                        ? vtm_set_admittance(T, VTM_W_ALPHA, P->W, 0, nullptr)
                        : vtm_set_admittance(T, VTM_W_LINE, 0.0, 0, P->port_W.data());
    if (st == VTM_OK) st = vtm_factor(T);
    if (st != VTM_OK) {
      vtm_destroy(T);
      return st;
    }
    P->transposed = T;
  }
  P->transposed->opts = P->opts;
  return solve_entry(P->transposed, g, lam, nrhs, tol, info);
}

extern "C" vtm_status vtm_residual_norm(vtm_plan_t P, const double* x, const double* b, int64_t nrhs,
                                        double* rel) {
  if (!P || !x || !b || !rel || nrhs <= 0) return VTM_EINVAL;
  cudaSetDevice(P->device);
  const int64_t count = P->n * nrhs;
  Staged Sx, Sb;
  VTM_TRY(stage(P, x, nullptr, count, Sx, 0));
  VTM_TRY(stage(P, b, nullptr, count, Sb, 1));
  vtm_status st = residual_norms(P, Sx.in_dev, Sb.in_dev, nrhs, rel);
  VTM_CUDA_TRY(cudaStreamSynchronize(P->stream));
  return st;
}
