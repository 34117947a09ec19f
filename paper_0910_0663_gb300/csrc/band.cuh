// Warp-level solves with the band factors of K_P.
//
// Storage (written by band_factor_kernel), column j of the tile's band:
//   Lc[j][0] = 1/L(j,j),  Lc[j][a] = L(j+a, j)/L(j,j)   a = 1..bw
//   Uc[j][0] = 1/U(j,j),  Uc[j][b] = U(j-b, j)/U(j,j)   b = 1..bw
// With the multipliers pre-divided by the pivot, each step of a column sweep
// is one FMA per lane on a value no earlier lane has to rescale:
//   forward:  v(j+a) -= Lc[j][a] v(j),  then y(j) = v(j) Lc[j][0]
//   backward: v(j-b) -= Uc[j][b] v(j),  then x(j) = v(j) Uc[j][0]
// (the final scalings are one parallel pass each).  This keeps the serial
// dependency chain at one shared-memory round trip per row and spends the
// FP64 pipe only on the band FMAs.
#pragma once

namespace vtm {

template <class FT>
__device__ __forceinline__ void warp_scale_pass(FT* v, int n, const FT* __restrict__ col0, int B) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int j = lane; j < n; j += 32) v[j] *= __ldg(col0 + (size_t)j * B);
  __syncwarp();
}

// Plain column sweeps (any bandwidth).
template <class FT>
__device__ __forceinline__ void warp_band_solve_plain(FT* v, int n, int bw, const FT* __restrict__ lc,
                                                      const FT* __restrict__ uc, int start) {
  const int lane = threadIdx.x & 31;
  const int B = bw + 1;
  for (int j = start; j < n; ++j) {
    const FT* col = lc + (size_t)j * B;
    const FT u = v[j];
    const int m = min(bw, n - 1 - j);
    for (int a = lane + 1; a <= m; a += 32) v[j + a] -= __ldg(col + a) * u;
    __syncwarp();
  }
  warp_scale_pass(v, n, lc, B);
  for (int j = n - 1; j >= 0; --j) {
    const FT* col = uc + (size_t)j * B;
    const FT u = v[j];
    const int m = min(bw, j);
    for (int b = lane + 1; b <= m; b += 32) v[j - b] -= __ldg(col + b) * u;
    __syncwarp();
  }
  warp_scale_pass(v, n, uc, B);
}

// The same sweeps with the multipliers of column j + D loaded while column j
// is applied (lane owns entries a = lane + 1 + 32 q, q < Q; needs bw <= 32 Q).
template <int Q, int D, class FT>
__device__ __forceinline__ void warp_band_solve_pf(FT* v, int n, int bw, const FT* __restrict__ lc,
                                                   const FT* __restrict__ uc, int start) {
  const int lane = threadIdx.x & 31;
  const int B = bw + 1;
  FT buf[D][Q];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int j = start + d;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int a = lane + 1 + 32 * q;
      buf[d][q] = (j < n && a <= min(bw, n - 1 - j)) ? __ldg(lc + (size_t)j * B + a) : FT(0);
    }
  }
  for (int j0 = start; j0 < n; j0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = j0 + d;
      if (j < n) {
        const FT u = v[j];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int a = lane + 1 + 32 * q;
          if (a <= min(bw, n - 1 - j)) v[j + a] -= buf[d][q] * u;
        }
        __syncwarp();
        const int jn = j + D;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int a = lane + 1 + 32 * q;
          buf[d][q] = (jn < n && a <= min(bw, n - 1 - jn)) ? __ldg(lc + (size_t)jn * B + a) : FT(0);
        }
      }
    }
  }
  warp_scale_pass(v, n, lc, B);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int j = n - 1 - d;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int b = lane + 1 + 32 * q;
      buf[d][q] = (j >= 0 && b <= min(bw, j)) ? __ldg(uc + (size_t)j * B + b) : FT(0);
    }
  }
  for (int j0 = n - 1; j0 >= 0; j0 -= D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = j0 - d;
      if (j >= 0) {
        const FT u = v[j];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int b = lane + 1 + 32 * q;
          if (b <= min(bw, j)) v[j - b] -= buf[d][q] * u;
        }
        __syncwarp();
        const int jn = j - D;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int b = lane + 1 + 32 * q;
          buf[d][q] = (jn >= 0 && b <= min(bw, jn)) ? __ldg(uc + (size_t)jn * B + b) : FT(0);
        }
      }
    }
  }
  warp_scale_pass(v, n, uc, B);
}

// K_P^-1 v in place (v in shared or global memory, one warp).  Deeper
// prefetch than 16 rows costs more registers than it gains: occupancy drops
// below one warp per tile and SM slot.
template <class FT>
__device__ __forceinline__ void warp_band_solve_any(FT* v, int n, int bw, const FT* __restrict__ lc,
                                                    const FT* __restrict__ uc, int start) {
  if (bw <= 32) warp_band_solve_pf<1, 16>(v, n, bw, lc, uc, start);
  else if (bw <= 64) warp_band_solve_pf<2, 12>(v, n, bw, lc, uc, start);
  else if (bw <= 128) warp_band_solve_pf<4, 8>(v, n, bw, lc, uc, start);
  else warp_band_solve_plain(v, n, bw, lc, uc, start);
}

}  // namespace vtm
