// Channel form of the sweep: torn lines plus lagged couplings (cut entries
// that are not branches, e.g. controlled sources), and block Jacobi.
//
// Per sub-circuit P, sweep k (Sec. VI, Eq. 11 with the lagged couplings of
// the cut moved to the right-hand side with one sweep of delay, reading R2):
//   K_P x_P = b_P + sum_ports beta_s w_in(s) e_l(s) - sum_lag rho_q z_q e_i(q)
// with z_q = x_j(q) of the previous sweep (read from tile Q).  Condensed:
//   [w_out; y] = E_P [w_in; z] + [c; y0],   y = the node voltages of P that
// other tiles' lagged entries read ("probes").  E_P is built column by column
// from banded solves: input a with right-hand side sigma_a e_loc(a)
// (sigma = beta for a port, -rho for a lagged entry) gives, for outputs o,
//   E(o, a) = scale_o y(loc(o)) + [a, o are the same port] (W - 2g)/(W + 2g),
//   scale = 2 W beta for a port output, 1 for a probe.
// Block Jacobi is the case without lines: every cut entry is lagged and
// K_P = A_PP, x_P^k = A_PP^-1 (b_P - sum_Q A_PQ x_Q^(k-1)) (Sec. X).
//
// Residual of sweep k at row i: torn branch s (twin t):
//   ((W - 2g) u_s + (W + 2g) u_t - w_in(s) - w_in(t)) / 2  (waves carried as w / d),
// lagged entry q: rho_q (z_q - x_j^k)   (z_q = x_j^(k-1) was used).
#include <algorithm>
#include <cmath>

#include "band.cuh"
#include "vtm_internal.h"

namespace vtm {

// one warp per input channel: column `a` of E_P (stored as row a of E_P^T)
__global__ void build_general_kernel(const int32_t* __restrict__ node_off,
                                     const int32_t* __restrict__ bwv,
                                     const int64_t* __restrict__ band_off,
                                     const double* __restrict__ Lc, const double* __restrict__ Uc,
                                     const int32_t* __restrict__ in_tile,
                                     const int32_t* __restrict__ in_off,
                                     const int32_t* __restrict__ out_off,
                                     const int32_t* __restrict__ in_loc,
                                     const int32_t* __restrict__ in_own_out,
                                     const double* __restrict__ sigma,
                                     const int32_t* __restrict__ out_loc,
                                     const double* __restrict__ scale,
                                     const double* __restrict__ diag,
                                     const int64_t* __restrict__ E_off,
                                     const int32_t* __restrict__ E_ld, double* __restrict__ E) {
  extern __shared__ double y[];
  const int a = blockIdx.x;
  const int t = in_tile[a];
  const int n = node_off[t + 1] - node_off[t];
  const int lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) y[i] = 0.0;
  __syncwarp();
  const int la = in_loc[a];
  if (lane == 0) y[la] = sigma[a];
  __syncwarp();
  warp_band_solve_any(y, n, bwv[t], Lc + band_off[t], Uc + band_off[t], la);
  const int o0 = out_off[t], no = out_off[t + 1] - o0;
  double* row = E + E_off[t] + (size_t)(a - in_off[t]) * E_ld[t];
  const int own = in_own_out[a];
  for (int q = lane; q < no; q += 32) {
    const int o = o0 + q;
    double v = scale[o] * y[out_loc[o]];
    if (o == own) v += diag[o];
    row[q] = v;
  }
}

// c_o = scale_o x0(loc(o)) for every output (one block per tile)
__global__ void general_const_kernel(const int32_t* __restrict__ node_off,
                                     const int32_t* __restrict__ out_off,
                                     const int32_t* __restrict__ out_loc,
                                     const double* __restrict__ scale,
                                     const double* __restrict__ x0, double* __restrict__ c) {
  const int t = blockIdx.x;
  const int base = node_off[t];
  for (int o = out_off[t] + threadIdx.x; o < out_off[t + 1]; o += blockDim.x)
    c[o] = scale[o] * x0[base + out_loc[o]];
}

// v(row node) += sum of sigma_a * input_a over the inputs of that row (fixed order)
__global__ void general_inject_kernel(const int32_t* __restrict__ node_off,
                                      const int32_t* __restrict__ in_off,
                                      const int32_t* __restrict__ in_loc,
                                      const int32_t* __restrict__ res_perm,
                                      const uint8_t* __restrict__ res_run,
                                      const double* __restrict__ sigma,
                                      const double* __restrict__ in_state, double* __restrict__ v) {
  const int t = blockIdx.x;
  const int a0 = in_off[t], ni = in_off[t + 1] - a0;
  for (int k = threadIdx.x; k < ni; k += blockDim.x) {
    const int nr = res_run[a0 + k];
    if (!nr) continue;
    double acc = 0.0;
    for (int q = 0; q < nr; ++q) {
      const int a = a0 + res_perm[a0 + k + q];
      acc += sigma[a] * in_state[a];
    }
    v[node_off[t] + in_loc[a0 + res_perm[a0 + k]]] += acc;
  }
}

__device__ double gblock_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
  __syncthreads();
  return tot;
}

__device__ double gblock_sum_array(const double* __restrict__ a, int count) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += a[i];
  return gblock_sum(acc);
}

// One CTA per tile; the products run in KS groups of blockDim / KS threads:
// group g takes the inputs a = g, g + KS, ... of each output, the KS partial
// sums meet in shared memory and are added in group order (more loads in
// flight per output than one thread walking every input: a tile's E_P streams
// with only a few CTAs per SM).
template <int KS>
__global__ void __launch_bounds__(1024) general_sweep_kernel(
    const double* __restrict__ E, const int64_t* __restrict__ E_off, const int32_t* __restrict__ E_ld,
    const int32_t* __restrict__ in_off, const int32_t* __restrict__ out_off,
    const int32_t* __restrict__ in_src, const uint8_t* __restrict__ in_kind,
    const int32_t* __restrict__ in_twin, const int32_t* __restrict__ in_own_out,
    const double* __restrict__ coef, const double* __restrict__ dsc, const int32_t* __restrict__ res_perm,
    const uint8_t* __restrict__ res_run, const double* __restrict__ c, double* __restrict__ gin,
    double* __restrict__ gout, int64_t n_in, int64_t n_out, SweepCtrl* __restrict__ ctrl,
    double* __restrict__ partials, double* __restrict__ hist, int hist_len, int nparts) {
  extern __shared__ double sm[];
  __shared__ int s_k, s_flag;
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    s_k = *((volatile int*)&ctrl->k);
    s_flag = *((volatile int*)&ctrl->flag);
  }
  __syncthreads();
  if (s_flag) return;
  const int k = s_k;
  const int t = blockIdx.x;
  const int a0 = in_off[t], ni = in_off[t + 1] - a0;
  const int o0 = out_off[t], no = out_off[t + 1] - o0;
  double* vin = sm;       // [max_in]
  double* rc = sm + ni;   // [max_in]
  double* part = rc + ni;  // [KS][blockDim / KS]
  const double* pin = gin + (size_t)((k - 1) & 1) * n_in;
  const double* pout = gout + (size_t)((k - 1) & 1) * n_out;
  double* cin = gin + (size_t)(k & 1) * n_in;
  double* cout_ = gout + (size_t)(k & 1) * n_out;
  for (int q = threadIdx.x; q < ni; q += blockDim.x) {
    const int a = a0 + q;
    double vi = 0.0, r = 0.0;
    if (k > 1) {
      const double src = pout[in_src[a]];
      vi = src;
      if (in_kind[a] == 0) {
        const double wi_s = pin[a], wo_s = pout[in_own_out[a]];
        const double wi_t = pin[in_twin[a]], wo_t = src;
        // coef = g/W, dsc = d of the line (waves carried as w / d)
        const double Ss = wi_s + wo_s, St = wi_t + wo_t;
        r = 0.5 * dsc[a] * (0.5 * (Ss + St) - coef[a] * (Ss - St) - wi_s - wi_t);
      } else {
        r = coef[a] * (pin[a] - src);
      }
    }
    vin[q] = vi;
    rc[q] = r;
  }
  __syncthreads();
  double sq = 0.0;
  if (k > 1) {
    for (int q = threadIdx.x; q < ni; q += blockDim.x) {
      const int nr = res_run[a0 + q];
      if (nr) {
        double r = 0.0;
        for (int e = 0; e < nr; ++e) r += rc[res_perm[a0 + q + e]];
        sq += r * r;
      }
    }
  }
  const double tile_sq = gblock_sum(sq);
  const double* Eb = E + E_off[t];
  const int ld = E_ld[t];
  const int to = (int)blockDim.x / KS, g = threadIdx.x / to, ql = threadIdx.x % to;
  for (int q0 = 0; q0 < no; q0 += to) {
    const int q = q0 + ql;
    double acc = 0.0;
    if (q < no) {
#pragma unroll 4
      for (int a = g; a < ni; a += KS) acc += __ldg(Eb + (size_t)a * ld + q) * vin[a];
    }
    part[g * to + ql] = acc;
    __syncthreads();
    if (g == 0 && q < no) {
      double tot = c[o0 + q];
      for (int gg = 0; gg < KS; ++gg) tot += part[gg * to + ql];
      cout_[o0 + q] = tot;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < ni; q += blockDim.x) cin[a0 + q] = vin[q];
  if (threadIdx.x == 0) {
    partials[t] = tile_sq;
    __threadfence();
    s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double tot = gblock_sum_array(partials, nparts);
  if (threadIdx.x == 0) {
    int flag = 0;
    if (k > 1) {
      const int ks = k - 1;
      if (hist && ks <= hist_len) hist[ks - 1] = sqrt(tot / ctrl->bnorm2);
      if (ks == 1) ctrl->first_res2 = tot;
      ctrl->last_res2 = tot;
      if (!isfinite(tot) || (ks > 1 && tot > 1e12 * ctrl->first_res2 && ctrl->first_res2 > 0)) {
        flag = 3;
      } else if (tot <= ctrl->tol2) {
        flag = 1;
        ctrl->conv_sweep = ks;
      }
    }
    if (!flag && k >= ctrl->k_max) flag = 2;
    ctrl->counter = 0u;
    ctrl->k = k + 1;
    __threadfence();
    ctrl->flag = flag;
  }
}

vtm_status build_general_operators(vtm_plan_s* P) {
  cudaStream_t s = P->stream;
  const size_t bytes = std::max<int64_t>(P->E_elems, 8) * sizeof(double);
  VTM_TRY(dev_alloc(P->d_E, bytes));
  VTM_CUDA_TRY(cudaMemsetAsync(P->d_E.p, 0, bytes, s));
  if (P->n_in > 0) {
    const size_t smem = (size_t)P->max_nodes * sizeof(double);
    if (smem > 200 * 1024) {
      set_detail("vtm_factor: a sub-circuit with more than 25600 nodes has cut couplings");
      return VTM_EINVAL;
    }
    VTM_CUDA_TRY(cudaFuncSetAttribute(build_general_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    build_general_kernel<<<(unsigned)P->n_in, 32, smem, s>>>(
        P->tabs.node_off.as<int32_t>(), P->tabs.bw.as<int32_t>(), P->tabs.band_off.as<int64_t>(),
        P->d_Lc.as<double>(), P->d_Uc.as<double>(), P->d_in_tile.as<int32_t>(),
        P->d_in_off.as<int32_t>(), P->d_out_off.as<int32_t>(), P->d_in_loc.as<int32_t>(),
        P->d_in_own_out.as<int32_t>(), P->d_in_sigma.as<double>(), P->d_out_loc.as<int32_t>(),
        P->d_out_scale.as<double>(), P->d_out_diag.as<double>(), P->d_E_off.as<int64_t>(),
        P->d_E_ld.as<int32_t>(), P->d_E.as<double>());
    VTM_CUDA_TRY(cudaGetLastError());
  }
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  return VTM_OK;
}

vtm_status general_const(vtm_plan_s* P, const double* x0) {
  general_const_kernel<<<P->nparts, 128, 0, P->stream>>>(
      P->tabs.node_off.as<int32_t>(), P->d_out_off.as<int32_t>(), P->d_out_loc.as<int32_t>(),
      P->d_out_scale.as<double>(), x0, P->d_cg.as<double>());
  P->launch_count++;
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

vtm_status general_sweeps(vtm_plan_s* P, double bnorm2, double target2, int budget, double* hist,
                          int hist_len, int* sweep_out, int* flag_out) {
  cudaStream_t s = P->stream;
  SweepCtrl h{};
  h.k = 1;
  h.k_max = budget;
  h.tol2 = target2;
  h.bnorm2 = bnorm2 > 0 ? bnorm2 : 1.0;
  *P->h_ctrl = h;
  VTM_CUDA_TRY(cudaMemcpyAsync(P->d_ctrl.p, P->h_ctrl, sizeof(SweepCtrl), cudaMemcpyHostToDevice, s));
  VTM_CUDA_TRY(cudaMemsetAsync(P->d_gin.p, 0, 2 * std::max<int64_t>(P->n_in, 1) * sizeof(double), s));
  VTM_CUDA_TRY(cudaMemsetAsync(P->d_gout.p, 0, 2 * std::max<int64_t>(P->n_out, 1) * sizeof(double), s));
  // four groups of up to 256 threads per tile (one output each; eight groups
  // of 128 measured slower on the 1024^2 VCCS grid)
  constexpr int KS = 4;
  const int to = P->max_out <= 64 ? 64 : (P->max_out <= 128 ? 128 : 256);
  const int threads = KS * to;
  const size_t smem = (2 * (size_t)std::max(P->max_in, 1) + threads) * sizeof(double);
  if (smem > 48 * 1024)
    VTM_CUDA_TRY(cudaFuncSetAttribute(general_sweep_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  int launched = 0;
  while (true) {
    const int m = std::min(P->opts.check_every, budget + 1 - launched);
    VTM_CUDA_TRY(cudaEventRecord(P->evs0, s));
    for (int i = 0; i < m; ++i)
      general_sweep_kernel<KS><<<P->nparts, threads, smem, s>>>(
          P->d_E.as<double>(), P->d_E_off.as<int64_t>(), P->d_E_ld.as<int32_t>(),
          P->d_in_off.as<int32_t>(), P->d_out_off.as<int32_t>(), P->d_in_src.as<int32_t>(),
          P->d_in_kind.as<uint8_t>(), P->d_in_twin.as<int32_t>(), P->d_in_own_out.as<int32_t>(),
          P->d_in_coef.as<double>(), P->d_in_d.as<double>(), P->d_res_perm.as<int32_t>(),
          P->d_res_run.as<uint8_t>(),
          P->d_cg.as<double>(), P->d_gin.as<double>(), P->d_gout.as<double>(), P->n_in, P->n_out,
          P->d_ctrl.as<SweepCtrl>(), P->d_partials.as<double>(), hist, hist_len, P->nparts);
    VTM_CUDA_TRY(cudaGetLastError());
    launched += m;
    VTM_CUDA_TRY(cudaEventRecord(P->evs1, s));
    VTM_CUDA_TRY(cudaMemcpyAsync(P->h_ctrl, P->d_ctrl.p, sizeof(SweepCtrl), cudaMemcpyDeviceToHost, s));
    VTM_CUDA_TRY(cudaStreamSynchronize(s));
    float bms = 0.f;
    VTM_CUDA_TRY(cudaEventElapsedTime(&bms, P->evs0, P->evs1));
    P->sweep_ms += bms;
    P->sweep_launch_count += m;
    P->launch_count += m;
    if (P->h_ctrl->flag || launched > budget) break;
  }
  const SweepCtrl& r = *P->h_ctrl;
  *flag_out = r.flag;
  *sweep_out = r.flag == 1 ? r.conv_sweep : std::min(r.k - 1, budget);
  return VTM_OK;
}

vtm_status general_inject(vtm_plan_s* P, int sweep, double* v) {
  general_inject_kernel<<<P->nparts, 128, 0, P->stream>>>(
      P->tabs.node_off.as<int32_t>(), P->d_in_off.as<int32_t>(), P->d_in_loc.as<int32_t>(),
      P->d_res_perm.as<int32_t>(), P->d_res_run.as<uint8_t>(), P->d_in_sigma.as<double>(),
      P->d_gin.as<double>() + (size_t)(sweep & 1) * P->n_in, v);
  P->launch_count++;
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

}  // namespace vtm
