// Branch <-> nodal-matrix map of a resistor network (Sec. II, Eq. 1) and the
// gradients of a loss through A x = b.
//
// For A = sum_e g_e (e_i - e_j)(e_i - e_j)^T + diag(ground):
//   values:    a_ij = -sum of the branches between i and j,
//              a_ii = ground_i + sum of the branches at i (fixed summation order);
//   gradients: with lam = A^-T dL/dx,
//              dL/dg_e = -(lam_i - lam_j)(x_i - x_j),  dL/dground_i = -lam_i x_i,
//              summed over the right-hand-side columns.
#include <algorithm>
#include <numeric>

#include "vtm_internal.h"

struct vtm_netmap_s {
  int64_t n = 0, nnz = 0, nedges = 0;
  cudaStream_t stream = nullptr;
  vtm::DevBuf off_edge;   // int64[nnz]: branch of an off-diagonal position (-1: none / diagonal)
  vtm::DevBuf diag_pos;   // int64[n]: CSR position of a_ii
  vtm::DevBuf inc_off;    // int64[n+1]: branches incident to each node
  vtm::DevBuf inc_edge;   // int64[2 nedges]
  vtm::DevBuf ei, ej;     // int64[nedges]
};

namespace vtm {

__global__ void netmap_values_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                     const int64_t* __restrict__ off_edge,
                                     const int64_t* __restrict__ diag_pos,
                                     const int64_t* __restrict__ inc_off,
                                     const int64_t* __restrict__ inc_edge,
                                     const double* __restrict__ g, const double* __restrict__ ground,
                                     double* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int64_t e = off_edge[q];
      vals[q] = e >= 0 ? -g[e] : 0.0;
    }
    double d = ground ? ground[i] : 0.0;
    for (int64_t q = inc_off[i]; q < inc_off[i + 1]; ++q) d += g[inc_edge[q]];
    vals[diag_pos[i]] = d;
  }
}

__global__ void netmap_grad_kernel(int64_t n, int64_t nedges, const int64_t* __restrict__ ei,
                                   const int64_t* __restrict__ ej, const double* __restrict__ lam,
                                   const double* __restrict__ x, int64_t nrhs,
                                   double* __restrict__ grad_g, double* __restrict__ grad_ground) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nedges; e += stride) {
    const int64_t i = ei[e], j = ej[e];
    double acc = 0.0;
    for (int64_t r = 0; r < nrhs; ++r) {
      const double* l = lam + r * n;
      const double* xx = x + r * n;
      acc -= (l[i] - l[j]) * (xx[i] - xx[j]);
    }
    grad_g[e] = acc;
  }
  if (grad_ground) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      double acc = 0.0;
      for (int64_t r = 0; r < nrhs; ++r) acc -= lam[r * n + i] * x[r * n + i];
      grad_ground[i] = acc;
    }
  }
}

}  // namespace vtm

using namespace vtm;

template <class T>
static vtm_status to_host(std::vector<T>& h, const T* src, size_t count) {
  h.resize(count);
  if (!count) return VTM_OK;
  if (is_device_ptr(src)) {
    VTM_CUDA_TRY(cudaMemcpy(h.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::copy(src, src + count, h.begin());
  }
  return VTM_OK;
}

extern "C" vtm_status vtm_netmap_create(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                                        int64_t nedges, const int64_t* ei, const int64_t* ej,
                                        void* stream, vtm_netmap_t* out) {
  if (!out || n <= 0 || nedges < 0 || !rowptr || !colidx || (nedges > 0 && (!ei || !ej))) {
    set_detail("vtm_netmap_create: bad argument");
    return VTM_EINVAL;
  }
  *out = nullptr;
  std::vector<int64_t> rp, hi, hj;
  std::vector<int32_t> ci;
  VTM_TRY(to_host(rp, rowptr, (size_t)n + 1));
  const int64_t nnz = rp[n];
  VTM_TRY(to_host(ci, colidx, (size_t)nnz));
  VTM_TRY(to_host(hi, ei, (size_t)nedges));
  VTM_TRY(to_host(hj, ej, (size_t)nedges));
  auto find = [&](int64_t i, int64_t j) -> int64_t {
    const int32_t* b = ci.data() + rp[i];
    const int32_t* e = ci.data() + rp[i + 1];
    const int32_t* f = std::lower_bound(b, e, (int32_t)j);
    return (f != e && *f == j) ? (int64_t)(f - ci.data()) : -1;
  };
  std::vector<int64_t> off_edge(nnz, -1), diag(n, -1), inc_off(n + 1, 0), inc(2 * nedges);
  for (int64_t i = 0; i < n; ++i) {
    diag[i] = find(i, i);
    if (diag[i] < 0) {
      set_detail("vtm_netmap_create: missing diagonal entry in row " + std::to_string(i));
      return VTM_EINVAL;
    }
  }
  for (int64_t e = 0; e < nedges; ++e) {
    const int64_t i = hi[e], j = hj[e];
    if (i < 0 || j < 0 || i >= n || j >= n || i == j) {
      set_detail("vtm_netmap_create: branch " + std::to_string(e) + " has bad end nodes");
      return VTM_EINVAL;
    }
    const int64_t pij = find(i, j), pji = find(j, i);
    if (pij < 0 || pji < 0 || off_edge[pij] >= 0 || off_edge[pji] >= 0) {
      set_detail("vtm_netmap_create: branch " + std::to_string(e) +
                 " is not in the pattern or is parallel to another branch");
      return VTM_EINVAL;
    }
    off_edge[pij] = e;
    off_edge[pji] = e;
    inc_off[i + 1]++;
    inc_off[j + 1]++;
  }
  for (int64_t i = 0; i < n; ++i) inc_off[i + 1] += inc_off[i];
  std::vector<int64_t> fill(inc_off.begin(), inc_off.end() - 1);
  for (int64_t e = 0; e < nedges; ++e) {  // increasing branch index within each node
    inc[fill[hi[e]]++] = e;
    inc[fill[hj[e]]++] = e;
  }
  vtm_netmap_s* M = new (std::nothrow) vtm_netmap_s();
  if (!M) return VTM_ENOMEM;
  M->n = n;
  M->nnz = nnz;
  M->nedges = nedges;
  M->stream = static_cast<cudaStream_t>(stream);
  vtm_status st = VTM_OK;
  if ((st = upload(M->off_edge, off_edge, M->stream)) != VTM_OK ||
      (st = upload(M->diag_pos, diag, M->stream)) != VTM_OK ||
      (st = upload(M->inc_off, inc_off, M->stream)) != VTM_OK ||
      (st = upload(M->inc_edge, inc, M->stream)) != VTM_OK ||
      (st = upload(M->ei, hi, M->stream)) != VTM_OK || (st = upload(M->ej, hj, M->stream)) != VTM_OK) {
    vtm_netmap_destroy(M);
    return st;
  }
  if (cudaStreamSynchronize(M->stream) != cudaSuccess) {
    vtm_netmap_destroy(M);
    return VTM_ECUDA;
  }
  *out = M;
  return VTM_OK;
}

extern "C" vtm_status vtm_netmap_values(vtm_netmap_t M, const int64_t* rowptr, const double* g,
                                        const double* ground, double* vals) {
  if (!M || !rowptr || !g || !vals) return VTM_EINVAL;
  if (!is_device_ptr(rowptr) || !is_device_ptr(g) || !is_device_ptr(vals) ||
      (ground && !is_device_ptr(ground))) {
    set_detail("vtm_netmap_values: arrays must be device memory");
    return VTM_EINVAL;
  }
  const int grid = (int)std::min<int64_t>((M->n + 255) / 256, 152 * 8);
  netmap_values_kernel<<<std::max(grid, 1), 256, 0, M->stream>>>(
      M->n, rowptr, M->off_edge.as<int64_t>(), M->diag_pos.as<int64_t>(), M->inc_off.as<int64_t>(),
      M->inc_edge.as<int64_t>(), g, ground, vals);
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

extern "C" vtm_status vtm_netmap_gradient(vtm_netmap_t M, const double* lam, const double* x,
                                          int64_t nrhs, double* grad_g, double* grad_ground) {
  if (!M || !lam || !x || !grad_g || nrhs <= 0) return VTM_EINVAL;
  if (!is_device_ptr(lam) || !is_device_ptr(x) || !is_device_ptr(grad_g) ||
      (grad_ground && !is_device_ptr(grad_ground))) {
    set_detail("vtm_netmap_gradient: arrays must be device memory");
    return VTM_EINVAL;
  }
  const int64_t work = std::max(M->nedges, M->n);
  const int grid = (int)std::min<int64_t>((work + 255) / 256, 152 * 8);
  netmap_grad_kernel<<<std::max(grid, 1), 256, 0, M->stream>>>(M->n, M->nedges, M->ei.as<int64_t>(),
                                                              M->ej.as<int64_t>(), lam, x, nrhs,
                                                              grad_g, grad_ground);
  VTM_CUDA_TRY(cudaGetLastError());
  return VTM_OK;
}

extern "C" void vtm_netmap_destroy(vtm_netmap_t M) {
  if (!M) return;
  dev_free(M->off_edge);
  dev_free(M->diag_pos);
  dev_free(M->inc_off);
  dev_free(M->inc_edge);
  dev_free(M->ei);
  dev_free(M->ej);
  delete M;
}
