// Per sub-circuit factorisation and the voltage reflection matrices.
//
// K_P (the matrix of Eq. 11 after eliminating the twin rows, see vtm.h) is
// banded after the planner's reordering.  It is factored in FP64 by a
// right-looking band Cholesky (symmetric A) or band LU without pivoting,
// one CTA per sub-circuit, with the active (bw+1) x (bw+1) window in shared
// memory addressed circularly.  The factors are stored column-wise:
//   Lc[j][a] = L(j+a, j) / L(j, j), a = 1..bw;  Lc[j][0] = 1 / L(j, j)
//   Uc[j][b] = U(j-b, j) / U(j, j), b = 1..bw;  Uc[j][0] = 1 / U(j, j)
// (multipliers divided by the pivot: see band.cuh) so that both triangular
// solves are column sweeps with contiguous reads and one FMA per step.
//
// The reflection matrix of Sec. VIII, T_P = (W - S_P)(W + S_P)^-1, is built
// column by column from banded solves: column q of T_P is
//   T(s, q) = 2 W_s beta_s y_q(l(s)) + delta_sq (W_s - 2 g_s)/(W_s + 2 g_s),
//   K_P y_q = beta_q e_l(q),  beta = 2 g/(2 g + W)
// (W_s the admittance of the line of port s).  With waves carried as w / d
// (d_s = 1 for one W on every line, sqrt(W_s) otherwise) the stored operator
// is D^-1 T_P D: bout_s = 2 W_s beta_s / d_s and bin_q = beta_q d_q take the
// place of 2 W beta and beta, and it is symmetric whenever A is.
// It is stored transposed (row q of the block = column q of the operator)
// with rows padded to a multiple of 8 elements.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "band.cuh"
#include "ptx.h"
#include "vtm_internal.h"

namespace vtm {

// ---------------------------------------------------------------------------
// band factorisation
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap(int x, int B) { return x % B; }

template <bool kLU>
__global__ void __launch_bounds__(256) band_factor_kernel(const int32_t* __restrict__ node_off,
                                                          const int32_t* __restrict__ bwv,
                                                          const int64_t* __restrict__ band_off,
                                                          double* __restrict__ Lc,
                                                          double* __restrict__ Uc,
                                                          double* __restrict__ gwin, int Bmax,
                                                          int* __restrict__ err) {
  extern __shared__ double smem[];
  const int t = blockIdx.x;
  const int n = node_off[t + 1] - node_off[t];
  const int bw = bwv[t];
  const int B = bw + 1;
  double* lc = Lc + band_off[t];
  double* uc = Uc + band_off[t];
  double* win = gwin ? gwin + (size_t)t * Bmax * Bmax : smem;
  double* lcol = gwin ? smem : smem + (size_t)Bmax * Bmax;
  double* urow = lcol + Bmax;
  const int tid = threadIdx.x;
  // initial window: rows/cols 0..min(bw, n-1)
  const int r0 = min(B, n);
  for (int idx = tid; idx < r0 * r0; idx += blockDim.x) {
    int r = idx / r0, c = idx % r0;
    double v = 0.0;
    if (c <= r) v = lc[(size_t)c * B + (r - c)];
    else if (kLU) v = uc[(size_t)c * B + (c - r)];
    if (kLU || c <= r) win[wrap(r, B) * B + wrap(c, B)] = v;
  }
  __syncthreads();
  bool bad = false;
  for (int j = 0; j < n; ++j) {
    const int jm = wrap(j, B);
    const int m = min(bw, n - 1 - j);
    const double piv = win[jm * B + jm];
    double dinv;
    if (kLU) {
      bad = bad || !(fabs(piv) > 0.0) || !isfinite(piv);
      dinv = 1.0 / piv;
    } else {
      bad = bad || !(piv > 0.0) || !isfinite(piv);
      dinv = rsqrt(piv > 0.0 ? piv : 1.0);
    }
    for (int a = tid + 1; a <= m; a += blockDim.x) {
      lcol[a] = win[wrap(j + a, B) * B + jm] * dinv;
      if (kLU) urow[a] = win[jm * B + wrap(j + a, B)];
    }
    __syncthreads();
    // column j of the factors, multipliers divided by the pivot (see band.cuh);
    // column j of U was filled unscaled by the earlier steps and is scaled now
    for (int a = tid; a <= m; a += blockDim.x) {
      if (a == 0) {
        lc[(size_t)j * B] = kLU ? 1.0 : dinv;
        uc[(size_t)j * B] = dinv;
      } else {
        lc[(size_t)j * B + a] = kLU ? lcol[a] : lcol[a] * dinv;
        uc[(size_t)(j + a) * B + a] = kLU ? urow[a] : lcol[a];
      }
    }
    for (int b = tid + 1; b <= min(bw, j); b += blockDim.x) uc[(size_t)j * B + b] *= dinv;
    // rank-1 update of the trailing window
    if (kLU) {
      for (int idx = tid; idx < m * m; idx += blockDim.x) {
        int a = idx / m + 1, b = idx % m + 1;
        win[wrap(j + a, B) * B + wrap(j + b, B)] -= lcol[a] * urow[b];
      }
    } else {
      for (int idx = tid; idx < m * m; idx += blockDim.x) {
        int a = idx / m + 1, b = idx % m + 1;
        if (b <= a) win[wrap(j + a, B) * B + wrap(j + b, B)] -= lcol[a] * lcol[b];
      }
    }
    __syncthreads();
    // bring in row (and column) r = j + B, which no earlier step touched
    const int r = j + B;
    if (r < n) {
      for (int c = r - bw + tid; c <= r; c += blockDim.x) {
        win[wrap(r, B) * B + wrap(c, B)] = lc[(size_t)c * B + (r - c)];
        if (kLU && c < r) win[wrap(c, B) * B + wrap(r, B)] = uc[(size_t)r * B + (r - c)];
      }
    }
    __syncthreads();
  }
  if (bad && tid == 0) atomicMax(err, t + 1);
}

vtm_status factor_tiles(vtm_plan_s* P) {
  cudaStream_t s = P->stream;
  const int Bmax = P->max_bw + 1;
  size_t win_bytes = (size_t)Bmax * Bmax * sizeof(double);
  size_t vec_bytes = 2 * (size_t)Bmax * sizeof(double);
  DevBuf gwin;
  bool use_smem = win_bytes + vec_bytes <= 200 * 1024;
  size_t smem = use_smem ? win_bytes + vec_bytes : vec_bytes;
  if (!use_smem) VTM_TRY(dev_alloc(gwin, (size_t)P->nparts * win_bytes));
  VTM_CUDA_TRY(cudaMemsetAsync(P->d_err.p, 0, sizeof(int), s));
  int threads = Bmax <= 40 ? 128 : 256;
  if (P->symmetric) {
    VTM_CUDA_TRY(cudaFuncSetAttribute(band_factor_kernel<false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    band_factor_kernel<false><<<P->nparts, threads, smem, s>>>(
        P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(),
        P->d_Lc.as<double>(), P->d_Uc.as<double>(), gwin.as<double>(), Bmax, P->d_err.as<int>());
  } else {
    VTM_CUDA_TRY(cudaFuncSetAttribute(band_factor_kernel<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    band_factor_kernel<true><<<P->nparts, threads, smem, s>>>(
        P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(),
        P->d_Lc.as<double>(), P->d_Uc.as<double>(), gwin.as<double>(), Bmax, P->d_err.as<int>());
  }
  VTM_CUDA_TRY(cudaGetLastError());
  int herr = 0;
  VTM_CUDA_TRY(cudaMemcpyAsync(&herr, P->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  dev_free(gwin);
  if (herr) {
    set_detail("vtm_factor: bad pivot in sub-circuit " + std::to_string(herr - 1));
    return VTM_ESINGULAR;
  }
  return VTM_OK;
}

// ---------------------------------------------------------------------------
// banded solves (one warp per right-hand side)
// ---------------------------------------------------------------------------

// Solve K_P x = v for every tile, in place in the permuted vector v
// (one warp per (tile, column)); columns are `stride` apart.
template <class FT>
__global__ void band_solve_tiles_kernel(const int32_t* __restrict__ node_off,
                                        const int32_t* __restrict__ bwv,
                                        const int64_t* __restrict__ band_off,
                                        const FT* __restrict__ Lc, const FT* __restrict__ Uc,
                                        FT* __restrict__ v, int64_t stride, int nparts,
                                        int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FT* smem = reinterpret_cast<FT*>(smem_raw);
  const int t = blockIdx.x % nparts;
  const int col = blockIdx.x / nparts;
  const int off = node_off[t];
  const int n = node_off[t + 1] - off;
  FT* vg = v + (size_t)col * stride + off;
  const int lane = threadIdx.x;
  if (use_smem) {
    for (int i = lane; i < n; i += 32) smem[i] = vg[i];
    __syncwarp();
    warp_band_solve_any(smem, n, bwv[t], Lc + band_off[t], Uc + band_off[t], 0);
    for (int i = lane; i < n; i += 32) vg[i] = smem[i];
  } else {
    warp_band_solve_any(vg, n, bwv[t], Lc + band_off[t], Uc + band_off[t], 0);
  }
}

// The same solve with the factor columns streamed through a shared-memory
// ring: chunks of kBC columns (contiguous in the band storage) are copied by
// 4- or 8-byte cp.async, kBS chunks ahead of the row being eliminated, so the
// serial row chain of a warp reads its multipliers from shared memory instead
// of waiting on HBM (deeper register prefetch cost occupancy).  The final
// scalings are folded in: y(j) = v(j) Lc[j][0] once row j's updates are out.
// Measured on the 2048^2 power grid: FP32 475 us per solve against 700 us
// for the register-prefetch kernel; FP64 1.8 ms against 1.3 ms (fewer
// resident warps for the FP64 pipe), so FP64 keeps the other kernel.
constexpr int kBC = 16;  // columns per chunk
constexpr int kBS = 4;   // chunks in flight

template <class FT>
__device__ __forceinline__ void cp_async_elem(FT* smem, const FT* gmem) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(FT) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(a), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(gmem) : "memory");
}

template <class FT, int Q>
__global__ void __launch_bounds__(32) band_solve_stream_kernel(
    const int32_t* __restrict__ node_off, const int32_t* __restrict__ bwv,
    const int64_t* __restrict__ band_off, const FT* __restrict__ Lc, const FT* __restrict__ Uc,
    FT* __restrict__ v, int64_t stride, int nparts, int n_max, int B_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FT* x = reinterpret_cast<FT*>(smem_raw);
  FT* ring = x + ((n_max + 1) & ~1);
  const int t = blockIdx.x % nparts;
  const int col = blockIdx.x / nparts;
  const int off = node_off[t];
  const int n = node_off[t + 1] - off;
  const int bw = bwv[t];
  const int B = bw + 1;
  const int lane = threadIdx.x;
  FT* vg = v + (size_t)col * stride + off;
  const FT* lc = Lc + band_off[t];
  const FT* uc = Uc + band_off[t];
  for (int i = lane; i < n; i += 32) x[i] = vg[i];
  const int nch = (n + kBC - 1) / kBC;
  // chunk c of a pass: columns [c kBC, ...) forward, [n - (c+1) kBC, ...) backward
  auto issue = [&](const FT* base, int c, bool fwd) {
    if (c < nch) {
      const int j0 = fwd ? c * kBC : max(0, n - (c + 1) * kBC);
      const int j1 = fwd ? min(n, (c + 1) * kBC) : n - c * kBC;
      FT* dst = ring + (size_t)(c % kBS) * kBC * B_max;
      const FT* src = base + (size_t)j0 * B;
      const int cnt = (j1 - j0) * B;
      for (int e = lane; e < cnt; e += 32) cp_async_elem(dst + e, src + e);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    const FT* base = fwd ? lc : uc;
    for (int c = 0; c < kBS; ++c) issue(base, c, fwd);
    __syncwarp();
    for (int c = 0; c < nch; ++c) {
      asm volatile("cp.async.wait_group %0;" ::"n"(kBS - 1) : "memory");
      __syncwarp();
      const FT* stg = ring + (size_t)(c % kBS) * kBC * B_max;
      const int j0 = fwd ? c * kBC : max(0, n - (c + 1) * kBC);
      const int j1 = fwd ? min(n, (c + 1) * kBC) : n - c * kBC;
      for (int q = 0; q < j1 - j0; ++q) {
        const int j = fwd ? j0 + q : j1 - 1 - q;
        const FT* colj = stg + (size_t)(j - j0) * B;
        const FT u = x[j];
        const int m = fwd ? min(bw, n - 1 - j) : min(bw, j);
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          const int a = lane + 1 + 32 * r;
          if (a <= m) {
            if (fwd) x[j + a] -= colj[a] * u;
            else x[j - a] -= colj[a] * u;
          }
        }
        if (lane == 0) x[j] = u * colj[0];
        __syncwarp();
      }
      issue(base, c + kBS, fwd);  // this stage is read: refill it
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) vg[i] = x[i];
}

// Band solves of bandwidth <= 32 in 32-row blocks held in registers: lane l
// keeps row J + l of the current block and row J + 32 + l of the next one.
// Step q of a block broadcasts u = v(J + q) from lane q (a shuffle, the only
// serial link of the row chain) and every lane applies one multiplier of
// column J + q: lanes l > q to their own row (offset l - q), lanes l <= q to
// the next block's row (offset 32 + l - q, still within the band).  Each
// lane therefore reads exactly one multiplier per column, loaded kPfD (FP32)
// or kPfD / 2 (FP64) columns ahead into a rotating register buffer.  The updates of every row
// arrive in increasing column order, as in warp_band_solve_pf, so the
// results are those of the column sweep.  The backward pass runs the same
// steps in reversed row order over Uc; y lives in shared memory between the
// passes.
constexpr int kPfD = 16;  // columns of multipliers in flight per lane

// Read-only loads and broadcasts as ordered (volatile) instructions: the
// prefetch distance is then what the code says (kPfD loads in flight), not
// the whole unrolled block hoisted into registers.
__device__ __forceinline__ float ld_nc_if(const float* p, bool ok) {
  float v = 0.f;
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q ld.global.nc.f32 %0, [%1];\n}"
               : "+f"(v) : "l"(p), "r"((int)ok));
  return v;
}
__device__ __forceinline__ double ld_nc_if(const double* p, bool ok) {
  double v = 0.0;
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q ld.global.nc.f64 %0, [%1];\n}"
               : "+d"(v) : "l"(p), "r"((int)ok));
  return v;
}
__device__ __forceinline__ float ld_nc(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_nc(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float shfl_idx_ordered(float x, int src) {
  float r;
  asm volatile("shfl.sync.idx.b32 %0, %1, %2, 0x1f, 0xffffffff;" : "=f"(r) : "f"(x), "r"(src));
  return r;
}
__device__ __forceinline__ double shfl_idx_ordered(double x, int src) {
  int lo = __double2loint(x), hi = __double2hiint(x);
  asm volatile("shfl.sync.idx.b32 %0, %0, %1, 0x1f, 0xffffffff;" : "+r"(lo) : "r"(src));
  asm volatile("shfl.sync.idx.b32 %0, %0, %1, 0x1f, 0xffffffff;" : "+r"(hi) : "r"(src));
  return __hiloint2double(hi, lo);
}

template <class FT, bool FWD>
__device__ __forceinline__ void band_pass_reg(const FT* __restrict__ colbase, int n, int bw, int B,
                                              const FT* __restrict__ vin, FT* ysm, FT* __restrict__ vout,
                                              int lane) {
  // pass coordinate j: row j (forward) or n - 1 - j (backward)
  auto src = [&](int j) -> FT { return j < n ? (FWD ? vin[j] : ysm[n - 1 - j]) : FT(0); };
  auto diag = [&](int j) -> FT { return j < n ? __ldg(colbase + (ptrdiff_t)(FWD ? j : n - 1 - j) * B) : FT(0); };
  // this lane's multiplier of pass column j = jb + q: offset a = l - q (own
  // row) or 32 + l - q (the next block's row), that is ((l - q - 1) mod 32) +
  // 1; it exists while a <= min(bw, n - 1 - j).  `ln` and `cs` are opaque
  // per-block copies of the lane and the column stride, so that what depends
  // only on (lane, q) is recomputed each block instead of being held in
  // registers for all 32 steps.
  auto load_col = [&](int jb, int q, int ln, int cs) -> FT {
    const int j = jb + q;
    const int a = ((ln - q - 1) & 31) + 1;
    const FT* c = colbase + (ptrdiff_t)(FWD ? j : n - 1 - j) * cs;
    return ld_nc_if(c + a, j < n && a <= min(bw, n - 1 - j));
  };
  constexpr int PD = sizeof(FT) == 4 ? kPfD : kPfD / 2;  // FP64: half the depth (registers)
  FT buf[PD];
#pragma unroll
  for (int d = 0; d < PD; ++d) buf[d] = load_col(0, d, lane, B);
  FT dg = diag(lane);
  FT xc = src(lane), xn = src(32 + lane);
  for (int J = 0; J < n; J += 32) {
    int ln = lane, cs = B;
    asm volatile("" : "+r"(ln), "+r"(cs));
    const FT dg_next = diag(J + 32 + lane);
    const FT x_after = src(J + 64 + lane);
    if (bw == 32 && J + 96 <= n) {
      // interior block of a full band: every multiplier loaded here exists.
      // Element of the multiplier of column jj for this lane, from colbase:
      // (jj or n - 1 - jj) 33 + a with a = ((l - jj - 1) mod 32) + 1; from
      // one column to the next a drops by one, wrapping from 1 to 32, so the
      // element moves by 32 or 64 (forward) or -34 or -2 (backward)
      const int jj0 = J + PD;
      int a = ((ln - jj0 - 1) & 31) + 1;
      int e = (FWD ? jj0 : n - 1 - jj0) * 33 + a;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const FT mq = buf[q % PD];
        buf[q % PD] = ld_nc(colbase + e);  // column J + q + PD
        const bool wrap = a == 1;
        e += FWD ? (wrap ? 64 : 32) : (wrap ? -2 : -34);
        a = wrap ? 32 : a - 1;
        const FT u = shfl_idx_ordered(xc, q);
        if (lane > q) xc -= mq * u;
        else xn -= mq * u;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const FT mq = buf[q % PD];
        buf[q % PD] = load_col(J, q + PD, ln, cs);  // column J + q + PD
        if (J + q < n) {
          const FT u = shfl_idx_ordered(xc, q);
          if (lane > q) xc -= mq * u;
          else xn -= mq * u;
        }
      }
    }
    if (J + lane < n) {
      const FT y = xc * dg;
      if (FWD) ysm[J + lane] = y;
      else vout[n - 1 - (J + lane)] = y;
    }
    xc = xn;
    xn = x_after;
    dg = dg_next;
  }
}

template <class FT>
__global__ void __launch_bounds__(32, 28) band_solve_reg_kernel(
    const int32_t* __restrict__ node_off, const int32_t* __restrict__ bwv,
    const int64_t* __restrict__ band_off, const FT* __restrict__ Lc, const FT* __restrict__ Uc,
    FT* __restrict__ v, int64_t stride, int nparts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FT* ysm = reinterpret_cast<FT*>(smem_raw);
  const int t = blockIdx.x % nparts;
  const int colr = blockIdx.x / nparts;
  const int off = node_off[t];
  const int n = node_off[t + 1] - off;
  const int bw = bwv[t];
  const int lane = threadIdx.x;
  FT* vg = v + (size_t)colr * stride + off;
  band_pass_reg<FT, true>(Lc + band_off[t], n, bw, bw + 1, vg, ysm, vg, lane);
  __syncwarp();
  band_pass_reg<FT, false>(Uc + band_off[t], n, bw, bw + 1, vg, ysm, vg, lane);
}

// The same register-blocked solve (FP32, half bandwidth <= 32) with the
// multipliers streamed through shared memory: each warp (one tile and column)
// keeps a ring of kRgS chunks of kRgC columns, filled by bulk copies that
// complete on one mbarrier per chunk slot, so that two chunks (about 4 KB) are
// on their way while the third is read -- twice the bytes in flight of the
// register prefetch, without its registers.  The forward results go back into
// v (global memory) instead of a shared-memory copy of the tile, which leaves
// room for 32 warps per SM.  Each lane applies the same multiplier of each
// column to the same row, in the same order, as band_pass_reg: the results are
// the same bits.  A chunk's copy starts at the 16-byte boundary below its
// first column (the FP32 factor arrays carry 64 bytes of tail padding for the
// rounded-up end of the last chunk).  Waits are bounded: a copy that never
// lands leaves the tile's column NaN (the refinement then reports a
// divergence) after a second bounded wait for the copies in flight.
constexpr int kRgC = 16;                  // columns per chunk
constexpr int kRgS = 3;                   // chunks per warp
constexpr int kRgStage = kRgC * 33 + 4;   // floats per chunk slot (532: a multiple of 4)
constexpr int kRgWarps = 4;               // warps per CTA
constexpr uint32_t kRgPolls = 1u << 24;   // mbarrier polls before giving up
constexpr size_t kRgSmem = (size_t)kRgWarps * (kRgS * kRgStage * sizeof(float) + kRgS * sizeof(uint64_t));

template <bool FWD>
__device__ __forceinline__ bool band_pass_ring(const float* __restrict__ colbase, int n, int bw, int B,
                                               float* v, float* ring, uint64_t* bars, uint32_t& par,
                                               int lane) {
  // pass coordinate j: row j (forward) or n - 1 - j (backward)
  auto src = [&](int j) -> float { return j < n ? v[FWD ? j : n - 1 - j] : 0.f; };
  auto diag = [&](int j) -> float {
    return j < n ? __ldg(colbase + (ptrdiff_t)(FWD ? j : n - 1 - j) * B) : 0.f;
  };
  const int nch = (n + kRgC - 1) / kRgC;
  // memory columns [mc0, mc1) of chunk c (pass columns [kRgC c, kRgC c + kRgC))
  auto first_col = [&](int c) { return FWD ? c * kRgC : n - min(n, c * kRgC + kRgC); };
  auto issue = [&](int c) {  // lane 0: chunk c into slot c mod kRgS
    const int mc0 = first_col(c);
    const int mc1 = FWD ? min(n, c * kRgC + kRgC) : n - c * kRgC;
    const uintptr_t a = reinterpret_cast<uintptr_t>(colbase + (size_t)mc0 * B);
    const uintptr_t a0 = a & ~(uintptr_t)15;
    const uint32_t bytes = (uint32_t)(((a - a0) + (size_t)(mc1 - mc0) * B * sizeof(float) + 15) & ~(size_t)15);
    uint64_t* bar = &bars[c % kRgS];
    mbar_arrive_expect_tx(bar, bytes);
    bulk_copy_g2s(ring + (c % kRgS) * kRgStage, reinterpret_cast<const void*>(a0), bytes, bar);
  };
  if (lane == 0) {
    fence_proxy_async_smem();  // the slots' earlier reads come before the copies
    for (int c = 0; c < kRgS && c < nch; ++c) issue(c);
  }
  float dg = diag(lane);
  float xc = src(lane), xn = src(32 + lane);
  for (int J = 0; J < n; J += 32) {
    const float dg_next = diag(J + 32 + lane);
    const float x_after = src(J + 64 + lane);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = (J >> 4) + h;
      if (c < nch) {
        const int sl = c % kRgS;
        if (!mbar_wait_bounded(&bars[sl], (par >> sl) & 1u, kRgPolls)) return false;
        par ^= 1u << sl;
        const float* st = ring + sl * kRgStage;
        const int mc0 = first_col(c);
        const int dl = (int)((reinterpret_cast<uintptr_t>(colbase + (size_t)mc0 * B) >> 2) & 3);
        if (bw == 32 && J + 96 <= n) {
          // interior block of a full band: every multiplier exists, and from
          // one column to the next the lane's element moves by 32 or 64
          // (forward) or -34 or -2 (backward) as its offset a wraps
          const int q0 = kRgC * h;
          int a = ((lane - q0 - 1) & 31) + 1;
          int e = dl + ((FWD ? J + q0 : n - 1 - (J + q0)) - mc0) * 33 + a;
#pragma unroll
          for (int qq = 0; qq < kRgC; ++qq) {
            const int q = q0 + qq;
            const float mq = st[e];
            const bool wrap = a == 1;
            e += FWD ? (wrap ? 64 : 32) : (wrap ? -2 : -34);
            a = wrap ? 32 : a - 1;
            const float u = shfl_idx_ordered(xc, q);
            if (lane > q) xc -= mq * u;
            else xn -= mq * u;
          }
        } else {
#pragma unroll
          for (int qq = 0; qq < kRgC; ++qq) {
            const int q = kRgC * h + qq, j = J + q;
            const int a = ((lane - q - 1) & 31) + 1;
            const int m = FWD ? j : n - 1 - j;
            const float mq = (j < n && a <= min(bw, n - 1 - j)) ? st[dl + (m - mc0) * B + a] : 0.f;
            if (j < n) {
              const float u = shfl_idx_ordered(xc, q);
              if (lane > q) xc -= mq * u;
              else xn -= mq * u;
            }
          }
        }
        __syncwarp();  // every lane is done with the slot
        if (lane == 0 && c + kRgS < nch) {
          fence_proxy_async_smem();
          issue(c + kRgS);
        }
      }
    }
    if (J + lane < n) v[FWD ? J + lane : n - 1 - (J + lane)] = xc * dg;
    xc = xn;
    xn = x_after;
    dg = dg_next;
  }
  return true;
}

__global__ void __launch_bounds__(32 * kRgWarps, 7) band_solve_ring_kernel(
    const int32_t* __restrict__ node_off, const int32_t* __restrict__ bwv,
    const int64_t* __restrict__ band_off, const float* __restrict__ Lc, const float* __restrict__ Uc,
    float* __restrict__ v, int64_t stride, int nparts, int nwork) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw) + warp * kRgS;
  float* ring = reinterpret_cast<float*>(smem_raw + kRgWarps * kRgS * sizeof(uint64_t)) +
                (size_t)warp * kRgS * kRgStage;
  const int g = blockIdx.x * kRgWarps + warp;
  if (g >= nwork) return;
  const int t = g % nparts;
  const int colr = g / nparts;
  const int off = node_off[t];
  const int n = node_off[t + 1] - off;
  const int bw = bwv[t];
  float* vg = v + (size_t)colr * stride + off;
  if (lane == 0) {
    for (int i = 0; i < kRgS; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t par = 0;
  bool ok = band_pass_ring<true>(Lc + band_off[t], n, bw, bw + 1, vg, ring, bars, par, lane);
  __syncwarp();  // y of every lane before the backward pass reads it
  if (ok) ok = band_pass_ring<false>(Uc + band_off[t], n, bw, bw + 1, vg, ring, bars, par, lane);
  if (!ok) {
    // a copy did not land: wait (bounded) for the slots still in flight,
    // then mark the column
    for (int i = 0; i < kRgS; ++i) mbar_wait_bounded(&bars[i], (par >> i) & 1u, kRgPolls);
    for (int i = lane; i < n; i += 32) vg[i] = __int_as_float(0x7fc00000);
  }
}

template <class FT>
static void launch_band_solve_t(vtm_plan_s* P, FT* v, const FT* Lc, const FT* Uc, int ncols,
                                int64_t stride, cudaStream_t s) {
  P->launch_count++;
  // FP32 only: the FP64 solve is bound by GB300's FP64 pipe either way (the
  // register-blocked form measured no faster for the 2048^2 power grid)
  if constexpr (sizeof(FT) == 4) {
    if (P->max_bw <= 32 && P->opts.band_solve == 0) {
      const int nwork = P->nparts * ncols;
      cudaFuncSetAttribute(band_solve_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRgSmem);
      band_solve_ring_kernel<<<(nwork + kRgWarps - 1) / kRgWarps, 32 * kRgWarps, kRgSmem, s>>>(
          P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(), Lc, Uc, v,
          stride, P->nparts, nwork);
      return;
    }
  }
  if (sizeof(FT) == 4 && P->max_bw <= 32) {
    const size_t smem = (size_t)std::max(P->max_nodes, 1) * sizeof(FT);
    if (smem <= 200 * 1024) {
      cudaFuncSetAttribute(band_solve_reg_kernel<FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      band_solve_reg_kernel<FT><<<P->nparts * ncols, 32, smem, s>>>(
          P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(), Lc, Uc, v,
          stride, P->nparts);
      return;
    }
  }
  // FP32 only: an FP64 solve is bound by GB300's FP64 pipe, where the
  // register-prefetch kernel (more resident warps) does better
  if (sizeof(FT) == 4 && P->max_bw <= 64) {
    const int B_max = P->max_bw + 1;
    const size_t smem = ((size_t)((P->max_nodes + 1) & ~1) + (size_t)kBS * kBC * B_max) * sizeof(FT);
    if (smem <= 200 * 1024) {
      auto kern = P->max_bw <= 32 ? band_solve_stream_kernel<FT, 1> : band_solve_stream_kernel<FT, 2>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<P->nparts * ncols, 32, smem, s>>>(P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(),
                                                P->tabs.band_off.as<int64_t>(), Lc, Uc, v, stride, P->nparts,
                                                P->max_nodes, B_max);
      return;
    }
  }
  size_t smem = (size_t)P->max_nodes * sizeof(FT);
  int use_smem = smem <= 200 * 1024;
  if (use_smem) {
    cudaFuncSetAttribute(band_solve_tiles_kernel<FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  } else {
    smem = 0;
  }
  band_solve_tiles_kernel<FT><<<P->nparts * ncols, 32, smem, s>>>(
      P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(), Lc,
      Uc, v, stride, P->nparts, use_smem);
}

void launch_band_solve(vtm_plan_s* P, double* v, int ncols, int64_t stride, cudaStream_t s) {
  launch_band_solve_t<double>(P, v, P->d_Lc.as<double>(), P->d_Uc.as<double>(), ncols, stride, s);
}

void launch_band_solve32(vtm_plan_s* P, float* v, int ncols, int64_t stride, cudaStream_t s) {
  launch_band_solve_t<float>(P, v, P->d_Lc32.as<float>(), P->d_Uc32.as<float>(), ncols, stride, s);
}

// ---------------------------------------------------------------------------
// reflection matrices
// ---------------------------------------------------------------------------

// One warp per port q: solve K_P y = beta_q e_l(q) and write row q of T_P^T.
__global__ void build_reflection_kernel(const int32_t* __restrict__ node_off,
                                        const int32_t* __restrict__ bwv,
                                        const int64_t* __restrict__ band_off,
                                        const double* __restrict__ Lc, const double* __restrict__ Uc,
                                        const int32_t* __restrict__ port_off,
                                        const int32_t* __restrict__ port_tile,
                                        const int32_t* __restrict__ port_loc,
                                        const double* __restrict__ bin,
                                        const double* __restrict__ bout,
                                        const double* __restrict__ rho,
                                        const int64_t* __restrict__ T_off,
                                        const int32_t* __restrict__ T_ld,
                                        double* __restrict__ T) {
  extern __shared__ double y[];
  const int q = blockIdx.x;
  const int t = port_tile[q];
  const int n = node_off[t + 1] - node_off[t];
  const int p0 = port_off[t];
  const int p = port_off[t + 1] - p0;
  const int lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) y[i] = 0.0;
  __syncwarp();
  const int lq = port_loc[q];
  if (lane == 0) y[lq] = bin[q];
  __syncwarp();
  warp_band_solve_any(y, n, bwv[t], Lc + band_off[t], Uc + band_off[t], lq);
  double* row = T + T_off[t] + (size_t)(q - p0) * T_ld[t];
  for (int s = lane; s < p; s += 32) {
    const int ps = p0 + s;
    double v = bout[ps] * y[port_loc[ps]];
    if (ps == q) v += rho[ps];
    row[s] = v;
  }
}

__global__ void convert_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__device__ __forceinline__ void store_low(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void store_low(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }
__device__ __forceinline__ void store_low(__half* p, double v) { *p = __float2half_rn((float)v); }

// the full (unpacked) 16-bit copy of the reflection matrices
template <class H>
__global__ void convert_16_kernel(const double* __restrict__ a, H* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    store_low(b + i, a[i]);
}

// Packed symmetric copy of the reflection matrices (symmetric plans, scalar
// W: T_P is symmetric, Sec. VIII).  The two stored halves of T_P differ only
// by the rounding of their column solves; their mean is packed.
// (store_low above: the same rounding as the full 16-bit copies)

template <class TT>
__global__ void pack_sym_kernel(const double* __restrict__ T64, const TileDesc* __restrict__ tdesc,
                                TT* __restrict__ Tp) {
  const TileDesc d = tdesc[blockIdx.x];
  const int nb = (d.p + kSymB - 1) / kSymB;
  const int nel = nb * (nb + 1) / 2 * kSymB * kSymB;
  const double* Tb = T64 + d.T_off;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    int blk = e / (kSymB * kSymB);
    const int w = e % (kSymB * kSymB);
    int bi = 0;
    while (blk >= nb - bi) {
      blk -= nb - bi;
      ++bi;
    }
    const int bj = bi + blk;
    // FP32 blocks are row-major; a 16-bit block keeps, at the 16 bytes of
    // lane l, row l/4 columns 4(l%4)..+3 then row l/4 + 8 (the sweep's order)
    int r = w / kSymB, q4 = w % kSymB;
    if (sizeof(TT) == 2) {
      const int l = w >> 3, e8 = w & 7;
      r = (l >> 2) + ((e8 >> 2) << 3);
      q4 = ((l & 3) << 2) + (e8 & 3);
    }
    const int s = bi * kSymB + r, q = bj * kSymB + q4;
    double v = 0.0;
    if (s < d.p && q < d.p) v = 0.5 * (Tb[(size_t)q * d.ld + s] + Tb[(size_t)s * d.ld + q]);
    store_low(Tp + d.Tp_off + e, v);
  }
}

// Packed double-float copy for the FP64-accurate sweep (kernel 12): the same
// blocks as the FP32 packed copy, each entry v = (T(s,q) + T(q,s))/2 kept as
// hi = rn32(v) in the block's first 256 floats and lo = rn32(v - hi) in its
// next 256 (a block is 512 floats; a tile's blocks start at 2 Tp_off).
__global__ void pack_sym_df_kernel(const double* __restrict__ T64, const TileDesc* __restrict__ tdesc,
                                   float* __restrict__ Tp) {
  const TileDesc d = tdesc[blockIdx.x];
  const int nb = (d.p + kSymB - 1) / kSymB;
  const int nel = nb * (nb + 1) / 2 * kSymB * kSymB;
  const double* Tb = T64 + d.T_off;
  float* out = Tp + 2 * d.Tp_off;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    int blk = e / (kSymB * kSymB);
    const int w = e % (kSymB * kSymB);
    const int nblk_before = blk;
    int bi = 0;
    while (blk >= nb - bi) {
      blk -= nb - bi;
      ++bi;
    }
    const int bj = bi + blk;
    const int s = bi * kSymB + w / kSymB, q = bj * kSymB + w % kSymB;
    double v = 0.0;
    if (s < d.p && q < d.p) v = 0.5 * (Tb[(size_t)q * d.ld + s] + Tb[(size_t)s * d.ld + q]);
    const float h = (float)v;
    out[(size_t)nblk_before * 2 * kSymB * kSymB + w] = h;
    out[(size_t)nblk_before * 2 * kSymB * kSymB + kSymB * kSymB + w] = (float)(v - (double)h);
  }
}

// the double-float copy serves FP64 plans of a symmetric A with at most 128
// ports per sub-circuit (kernel 12)
static bool packed_df_eligible(const vtm_plan_s* P) {
  return P->symmetric && !P->general && P->max_ports <= 8 * kSymB && !P->port_node.empty() &&
         P->opts.precision == VTM_PREC_FP64;
}

// Packed copies are kept for symmetric VTM plans whose sub-circuits have at
// most 256 ports (16 blocks a side), in the plan's low precision.
static bool packed_eligible(const vtm_plan_s* P) {
  return P->symmetric && !P->general && P->max_ports <= 16 * kSymB &&
         !P->port_node.empty() && P->opts.precision != VTM_PREC_FP64;
}

vtm_status build_reflections(vtm_plan_s* P) {
  cudaStream_t s = P->stream;
  const int64_t npt = (int64_t)P->port_node.size();
  const size_t Tbytes = std::max<int64_t>(P->T_elems, 8) * sizeof(double);
  VTM_TRY(dev_alloc(P->d_T64, Tbytes));
  VTM_CUDA_TRY(cudaMemsetAsync(P->d_T64.p, 0, Tbytes, s));
  if (npt > 0) {
    size_t smem = (size_t)P->max_nodes * sizeof(double);
    if (smem > 200 * 1024) {
      set_detail("vtm_factor: a sub-circuit with more than 25600 nodes has ports; use more parts");
      return VTM_EINVAL;
    }
    std::vector<int32_t> port_tile(npt);
    for (int32_t t = 0; t < P->nparts; ++t)
      for (int32_t q = P->port_off[t]; q < P->port_off[t + 1]; ++q) port_tile[q] = t;
    DevBuf d_pt;
    VTM_TRY(upload(d_pt, port_tile, s));
    VTM_CUDA_TRY(cudaFuncSetAttribute(build_reflection_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    build_reflection_kernel<<<(unsigned)npt, 32, smem, s>>>(
        P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(),
        P->d_Lc.as<double>(), P->d_Uc.as<double>(), P->tabs.port_off.as<int32_t>(),
        d_pt.as<int32_t>(), P->d_port_loc.as<int32_t>(), P->d_beta.as<double>(),
        P->d_bout.as<double>(), P->d_rho.as<double>(), P->tabs.T_off.as<int64_t>(),
        P->tabs.T_ld.as<int32_t>(), P->d_T64.as<double>());
    VTM_CUDA_TRY(cudaGetLastError());
    VTM_CUDA_TRY(cudaStreamSynchronize(s));
    dev_free(d_pt);
  }
  const int64_t ne = std::max<int64_t>(P->T_elems, 8);
  if (P->opts.precision == VTM_PREC_FP32) {
    VTM_TRY(dev_alloc(P->d_T32, ne * sizeof(float)));
    convert_f32_kernel<<<1216, 256, 0, s>>>(P->d_T64.as<double>(), P->d_T32.as<float>(), ne);
  } else if (P->opts.precision == VTM_PREC_BF16) {
    VTM_TRY(dev_alloc(P->d_T16, ne * sizeof(__nv_bfloat16)));
    convert_16_kernel<<<1216, 256, 0, s>>>(P->d_T64.as<double>(), P->d_T16.as<__nv_bfloat16>(), ne);
  } else if (P->opts.precision == VTM_PREC_FP16) {
    VTM_TRY(dev_alloc(P->d_T16, ne * sizeof(__half)));
    convert_16_kernel<<<1216, 256, 0, s>>>(P->d_T64.as<double>(), P->d_T16.as<__half>(), ne);
  }
  if (packed_eligible(P)) {
    const int64_t np = std::max<int64_t>(P->Tp_elems, 8);
    if (P->opts.precision == VTM_PREC_FP32) {
      VTM_TRY(dev_alloc(P->d_Tp32, np * sizeof(float)));
      pack_sym_kernel<float><<<P->nparts, 256, 0, s>>>(P->d_T64.as<double>(),
                                                       P->d_tdesc.as<TileDesc>(), P->d_Tp32.as<float>());
    } else if (P->opts.precision == VTM_PREC_BF16) {
      VTM_TRY(dev_alloc(P->d_Tp16, np * sizeof(__nv_bfloat16)));
      pack_sym_kernel<__nv_bfloat16><<<P->nparts, 256, 0, s>>>(
          P->d_T64.as<double>(), P->d_tdesc.as<TileDesc>(), P->d_Tp16.as<__nv_bfloat16>());
    } else {
      VTM_TRY(dev_alloc(P->d_Tp16, np * sizeof(__half)));
      pack_sym_kernel<__half><<<P->nparts, 256, 0, s>>>(P->d_T64.as<double>(), P->d_tdesc.as<TileDesc>(),
                                                        P->d_Tp16.as<__half>());
    }
  }
  if (packed_df_eligible(P)) {
    const int64_t np = std::max<int64_t>(P->Tp_elems, 8);
    VTM_TRY(dev_alloc(P->d_Tpdf, 2 * np * sizeof(float)));
    pack_sym_df_kernel<<<P->nparts, 256, 0, s>>>(P->d_T64.as<double>(), P->d_tdesc.as<TileDesc>(),
                                                 P->d_Tpdf.as<float>());
  } else if (P->d_Tpdf.p) {
    dev_free(P->d_Tpdf);  // the plan left FP64 (precision changed) or no longer qualifies
  }
  VTM_CUDA_TRY(cudaGetLastError());
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  return VTM_OK;
}

}  // namespace vtm

using namespace vtm;

extern "C" vtm_status vtm_factor(vtm_plan_t P) {
  if (!P) return VTM_EINVAL;
  cudaSetDevice(P->device);
  P->factored = false;
  // captured sweep batches refer to the operator buffers: rebuild them
  for (int i = 0; i < 4; ++i) {
    P->sweep_graph[i].reset();
    P->batch_graph[i].reset();
  }
  // the tiled copy of the tcgen05 batched sweep follows the factors
  dev_free(P->d_Ttc);
  P->tc_nitems = 0;
  // so do the blocked band-solve matrices
  dev_free(P->d_bk_Gf);
  dev_free(P->d_bk_Gb);
  P->bk_ready = false;
  // the band arrays hold K_P before the factorisation: re-assemble if a
  // previous factorisation overwrote them
  static_assert(sizeof(double) == 8, "");
  VTM_TRY(assemble_local(P));
  VTM_TRY(factor_tiles(P));
  if (P->opts.precision != VTM_PREC_FP64) {
    // FP32 copy of the factors for the right-hand-side preparation of the
    // inner (low-precision) solves
    const int64_t ne = std::max<int64_t>(P->band_elems, 8);
    // (+ 64 bytes: the bulk copies of the band solve round their last chunk up
    // to a 16-byte multiple)
    VTM_TRY(dev_alloc(P->d_Lc32, ne * sizeof(float) + 64));
    VTM_TRY(dev_alloc(P->d_Uc32, ne * sizeof(float) + 64));
    convert_f32_kernel<<<1216, 256, 0, P->stream>>>(P->d_Lc.as<double>(), P->d_Lc32.as<float>(), ne);
    convert_f32_kernel<<<1216, 256, 0, P->stream>>>(P->d_Uc.as<double>(), P->d_Uc32.as<float>(), ne);
    VTM_CUDA_TRY(cudaGetLastError());
  }
  if (P->general) {
    VTM_TRY(build_general_operators(P));
  } else {
    VTM_TRY(build_reflections(P));
  }
  P->factored = true;
  return VTM_OK;
}

extern "C" vtm_status vtm_get_reflection(vtm_plan_t P, int32_t part, double* T, int64_t cap,
                                         int32_t* p) {
  if (!P || part < 0 || part >= P->nparts) return VTM_EINVAL;
  if (!P->factored) return VTM_ENOTFACTORED;
  if (P->general) {
    set_detail("vtm_get_reflection: this plan carries lagged couplings; its tile operators "
               "include them and are not plain reflection matrices");
    return VTM_EINVAL;
  }
  const int32_t pp = P->port_off[part + 1] - P->port_off[part];
  if (p) *p = pp;
  if (!T) return VTM_OK;
  if (cap < (int64_t)pp * pp) return VTM_EINVAL;
  const int32_t ld = P->T_ld[part];
  std::vector<double> blk((size_t)pp * ld);
  if (pp > 0)
    VTM_CUDA_TRY(cudaMemcpy(blk.data(), P->d_T64.as<double>() + P->T_off[part],
                            blk.size() * sizeof(double), cudaMemcpyDeviceToHost));
  // back from the plan's wave scaling: T_P(s, q) = d_s [D^-1 T_P D](s, q) / d_q
  const int32_t p0 = P->port_off[part];
  for (int32_t q = 0; q < pp; ++q)
    for (int32_t s = 0; s < pp; ++s)
      T[(size_t)s * pp + q] = blk[(size_t)q * ld + s] * (P->port_d[p0 + s] / P->port_d[p0 + q]);
  return VTM_OK;
}

// Host decoding of one stored element of the low-precision copies.
static double stored_value(const void* base, int64_t i, int esize, int precision) {
  if (esize == 8) return static_cast<const double*>(base)[i];
  if (esize == 4) return static_cast<const float*>(base)[i];
  const uint16_t h = static_cast<const uint16_t*>(base)[i];
  if (precision == VTM_PREC_BF16) {
    const uint32_t u = (uint32_t)h << 16;  // BF16 is the upper half of an FP32
    float f;
    std::memcpy(&f, &u, 4);
    return f;
  }
  // FP16 (IEEE binary16): sign, 5-bit exponent (bias 15), 10-bit fraction
  const int sgn = h >> 15, ex = (h >> 10) & 31, fr = h & 1023;
  double v;
  if (ex == 0) v = std::ldexp((double)fr, -24);                 // subnormal
  else if (ex == 31) v = fr ? NAN : INFINITY;
  else v = std::ldexp(1.0 + fr / 1024.0, ex - 15);
  return sgn ? -v : v;
}

extern "C" vtm_status vtm_get_reflection_stored(vtm_plan_t P, int32_t part, double* T, int64_t cap,
                                                int32_t* p, int32_t* stored, int32_t* packed) {
  if (!P || part < 0 || part >= P->nparts) return VTM_EINVAL;
  if (!P->factored) return VTM_ENOTFACTORED;
  if (P->general) {
    set_detail("vtm_get_reflection_stored: this plan carries lagged couplings");
    return VTM_EINVAL;
  }
  cudaSetDevice(P->device);
  const int prec = P->opts.precision;
  const int32_t pp = P->port_off[part + 1] - P->port_off[part];
  const bool is_df = prec == VTM_PREC_FP64 && P->d_Tpdf.p;
  const bool is_packed = ((P->d_Tp32.p || P->d_Tp16.p) && prec != VTM_PREC_FP64) || is_df;
  const int esize = prec == VTM_PREC_FP64 ? 8 : prec == VTM_PREC_FP32 ? 4 : 2;
  if (p) *p = pp;
  if (stored) *stored = esize;
  if (packed) *packed = is_packed ? 1 : 0;
  if (!T) return VTM_OK;
  if (cap < (int64_t)pp * pp) return VTM_EINVAL;
  if (pp == 0) return VTM_OK;
  const int32_t p0 = P->port_off[part];
  auto unscale = [&](int32_t s, int32_t q) { return P->port_d[p0 + s] / P->port_d[p0 + q]; };
  if (is_packed) {
    // blocks (bi <= bj) row-major over (bi, bj); an FP32 block is row-major, a
    // 16-bit block keeps at the 16 bytes of lane l its row l/4, columns
    // 4(l%4)..+3, then row l/4 + 8 (the layout pack_sym_kernel writes)
    const int nb = (pp + kSymB - 1) / kSymB;
    const int64_t nel = (int64_t)nb * (nb + 1) / 2 * kSymB * kSymB;
    std::vector<unsigned char> raw((size_t)nel * esize);
    const unsigned char* src = static_cast<const unsigned char*>(
        is_df ? P->d_Tpdf.p : esize == 4 ? P->d_Tp32.p : P->d_Tp16.p);
    VTM_CUDA_TRY(cudaMemcpy(raw.data(), src + (size_t)P->Tp_off[part] * esize, raw.size(),
                            cudaMemcpyDeviceToHost));
    // double-float blocks: 256 hi floats, then 256 lo floats
    auto df_value = [&](int64_t e) {
      const float* f = reinterpret_cast<const float*>(raw.data());
      const int64_t blk = e / (kSymB * kSymB), w = e % (kSymB * kSymB);
      return (double)f[blk * 2 * kSymB * kSymB + w] + (double)f[blk * 2 * kSymB * kSymB + kSymB * kSymB + w];
    };
    int64_t e = 0;
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj)
        for (int w = 0; w < kSymB * kSymB; ++w, ++e) {
          int r = w / kSymB, q4 = w % kSymB;
          if (esize == 2) {
            const int l = w >> 3, e8 = w & 7;
            r = (l >> 2) + ((e8 >> 2) << 3);
            q4 = ((l & 3) << 2) + (e8 & 3);
          }
          const int s = bi * kSymB + r, q = bj * kSymB + q4;
          if (s >= pp || q >= pp) continue;
          const double v = is_df ? df_value(e) : stored_value(raw.data(), e, esize, prec);
          T[(size_t)s * pp + q] = v * unscale(s, q);
          T[(size_t)q * pp + s] = v * unscale(q, s);
        }
    return VTM_OK;
  }
  // full copy: per tile a p x ld block of T_P^T (row q = column q of T_P)
  const int32_t ld = P->T_ld[part];
  std::vector<unsigned char> raw((size_t)pp * ld * esize);
  const unsigned char* src = static_cast<const unsigned char*>(
      esize == 8 ? P->d_T64.p : esize == 4 ? P->d_T32.p : P->d_T16.p);
  VTM_CUDA_TRY(cudaMemcpy(raw.data(), src + (size_t)P->T_off[part] * esize, raw.size(),
                          cudaMemcpyDeviceToHost));
  for (int32_t q = 0; q < pp; ++q)
    for (int32_t s = 0; s < pp; ++s)
      T[(size_t)s * pp + q] = stored_value(raw.data(), (int64_t)q * ld + s, esize, prec) * unscale(s, q);
  return VTM_OK;
}
