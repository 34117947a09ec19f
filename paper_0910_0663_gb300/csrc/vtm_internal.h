// Internal declarations shared by the translation units of libvtm.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vtm.h"

namespace vtm {

// Thread-local detail message for vtm_last_error_detail().
void set_detail(const std::string& msg);

#define VTM_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ::vtm::set_detail(std::string(#expr) + ": " + cudaGetErrorString(e_));      \
      return (e_ == cudaErrorMemoryAllocation) ? VTM_ENOMEM : VTM_ECUDA;          \
    }                                                                             \
  } while (0)

#define VTM_TRY(expr)                         \
  do {                                        \
    vtm_status s_ = (expr);                   \
    if (s_ != VTM_OK) return s_;              \
  } while (0)

// A device allocation released by the plan.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Device-side control block of one solve (one per plan).
struct SweepCtrl {
  int k;               // index of the sweep the next launch runs (1-based)
  int flag;            // 0 running, 1 converged, 2 sweep limit, 3 diverged, 4 stalled
  unsigned counter;    // CTAs of the current launch that finished
  int conv_sweep;      // sweep whose residual met the tolerance
  int k_max;           // last sweep allowed
  int best_k;          // sweep with the smallest residual so far
  int stall;           // sweeps without a 10% improvement that end the run (0 = never)
  unsigned ticket;     // unused (kept for the layout; the one-warp-per-tile sweeps count
                       // their sweeps per CTA after the block)
  double best_res2;    // smallest squared residual so far
  double tol2;         // (tol * ||b||)^2 for the residual test
  double bnorm2;       // ||b||^2 of the current right-hand side
  double first_res2;   // squared residual of sweep 1 (divergence guard)
  double last_res2;    // squared residual of the last completed sweep
};

// Per-launch-slot descriptor of a tile for the vector-load sweep kernel.
struct __align__(16) TileDesc {
  int32_t tile;
  int32_t p0;   // first port
  int32_t p;    // ports
  int32_t ld;   // row length of the T^T block
  int64_t T_off;
  int64_t Tp_off;  // packed symmetric form: first element of the tile's 16x16 blocks
};

// Two 16-bit storage types of the reflection matrices (BF16, FP16): a packed
// pair of them as two floats.
template <class H>
struct Pair16;
template <>
struct Pair16<__nv_bfloat16> {
  __device__ static float2 f2(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
  }
  __device__ static float f(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <>
struct Pair16<__half> {
  __device__ static float2 f2(uint32_t w) { return __half22float2(*reinterpret_cast<const __half2*>(&w)); }
  __device__ static float f(__half v) { return __half2float(v); }
};

// Relative residual at which an inner low-precision solve hands back to the
// FP64 refinement: a few units of the storage type's rounding of T_P (FP32
// 2^-24, FP16 2^-11, BF16 2^-8 relative), where its sweeps stop gaining.
inline double default_inner_tol(int precision) {
  switch (precision) {
    case VTM_PREC_FP32: return 1e-5;
    case VTM_PREC_FP16: return 1e-3;
    case VTM_PREC_BF16: return 3e-3;
    default: return 0.0;
  }
}

// Refinement safeguard.  Every FP64 refinement step around low-precision
// sweeps must cut ||b - A x|| by a fixed factor: 10x with FP32 sweeps, 2x
// with BF16/FP16 ones (whose T_P carries 2^-8 / 2^-11 relative rounding).
// Once ||r|| is within that factor of the target, a step must still cut it
// by 10%.  A step that gains less means the refinement has stalled (the
// inner problem is too ill-conditioned for the storage precision, or the
// inner tolerance is too loose) and the solve returns VTM_ENOCONV at once
// instead of spending its remaining steps.
inline double refinement_min_gain(int precision) {
  return precision == VTM_PREC_FP32 ? 10.0 : 2.0;
}
inline bool refinement_stalled(int precision, double r_prev, double r_now, double target) {
  if (precision == VTM_PREC_FP64) return false;
  const double gain = refinement_min_gain(precision);
  const double need = r_prev > gain * target ? r_prev / gain : 0.9 * r_prev;
  return !(r_now <= need);
}

// Packed symmetric reflection matrices: T_P padded to pp = 16 ceil(p/16),
// cut into 16x16 blocks, of which the upper triangle (bi <= bj) is stored,
// row-major over (bi, bj), each block row-major.
constexpr int kSymB = 16;

// Offsets and sizes describing one tile-contiguous operator family.
struct TileTables {
  DevBuf node_off;   // int32[nparts+1]: first permuted position of each tile
  DevBuf bw;         // int32[nparts]: half bandwidth
  DevBuf band_off;   // int64[nparts]: offset (doubles) of the tile's band columns
  DevBuf port_off;   // int32[nparts+1]
  DevBuf T_off;      // int64[nparts]: element offset of the tile's T^T block
  DevBuf T_ld;       // int32[nparts]: padded row length of the T^T block
  DevBuf order;      // int32[nparts]: launch order of tiles (largest p first)
};

}  // namespace vtm

namespace vtm {
// A captured batch of sweep launches (CUDA graph) and what it was made for.
// Captured sweep launches: `exec` replays check_every launches, `small` a
// quarter of that (the tail up to a hinted sweep count)
struct SweepGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraphExec_t small = nullptr;
  uint64_t key = 0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (small) cudaGraphExecDestroy(small);
    exec = small = nullptr;
    key = 0;
  }
};
}  // namespace vtm

struct vtm_plan_s {
  // problem description
  int64_t n = 0;
  int64_t nnz = 0;
  int32_t nparts = 0;
  double Zc = 1.0;
  double W = 1.0;  // admittance of every line while the choice is alpha I

  // characteristic admittance of the virtual lines (Sec. VIII), see
  // vtm_set_admittance; per port: W_s, the wave scaling d_s = sqrt(W_s/W_ref)
  // (1 for a scalar W) under which T_P stays symmetric, and the coefficients
  // the kernels use (beta d, 2 W beta / d, (W - 2g)/(W + 2g), (g/W, d))
  int w_kind = 0;
  double w_alpha = 0.0;
  int w_radius = 2;
  std::vector<double> w_user;
  std::vector<double> port_W, port_d;
  bool w_dirty = true;  // port_W to be recomputed from the current values
  vtm_opts opts{};
  cudaStream_t stream = nullptr;
  bool symmetric = true;
  bool factored = false;
  int device = 0;

  // host copies of the input (values change with vtm_set_values)
  std::vector<int64_t> h_rowptr;
  std::vector<int32_t> h_colidx;
  std::vector<double> h_vals;
  std::vector<int32_t> h_part;

  // tiles: permuted (tile-contiguous, band-ordered) numbering
  std::vector<int32_t> node_off;  // nparts+1
  std::vector<int32_t> perm;      // perm[pos] = node
  std::vector<int32_t> iperm;     // iperm[node] = pos
  std::vector<int32_t> bw;        // half bandwidth per tile
  std::vector<int64_t> band_off;  // offset (doubles) per tile: n_P * (bw+1)
  int64_t band_elems = 0;
  int32_t max_nodes = 0, max_bw = 0, max_ports = 0;

  // ports (two per torn branch), grouped by tile, then by (node, remote)
  std::vector<int32_t> port_off;     // nparts+1
  std::vector<int32_t> port_node;    // global node
  std::vector<int32_t> port_remote;  // node across the branch
  std::vector<int32_t> port_twin;    // twin port
  std::vector<int32_t> port_loc;     // permuted position - tile start of the port node
  std::vector<int64_t> port_pos_ij;  // CSR position of a(node, remote) or -1
  std::vector<int64_t> port_pos_ji;  // CSR position of a(remote, node) or -1
  std::vector<double> port_g;        // branch conductance
  std::vector<uint8_t> port_run;     // ports left in this node's run (>=1) at a run start, else 0

  // lagged couplings (cut entries that are not branches), by row
  std::vector<int32_t> lag_i, lag_j;
  std::vector<int64_t> lag_pos;
  std::vector<double> lag_rho;

  // reflection-matrix layout
  std::vector<int32_t> T_ld;
  std::vector<int64_t> T_off;
  int64_t T_elems = 0;
  int64_t sum_p2 = 0;
  std::vector<int64_t> Tp_off;  // packed symmetric form (see TileDesc)
  int64_t Tp_elems = 0;
  int64_t sum_tri = 0;          // sum over tiles of p (p + 1) / 2

  // device copies
  vtm::TileTables tabs;
  vtm::DevBuf d_rowptr, d_colidx, d_vals;  // A for the FP64 residual
  vtm::DevBuf d_perm;                      // int32[n]
  vtm::DevBuf d_iperm;                     // int32[n] (batched solves)
  vtm::DevBuf d_Lc, d_Uc;                  // band factors (doubles)
  vtm::DevBuf d_Lc32, d_Uc32, d_v32;       // FP32 factor copies and work vector (inner solves)
  vtm::DevBuf d_v32b;                      // second FP32 work vector (the recovery's right-hand side)
  // A in ELL form for the single-column residual ([k][n] values and columns,
  // row lengths): 0 not built, 1 built, 2 rows too uneven (CSR kernel)
  vtm::DevBuf d_ell_val, d_ell_col, d_ell_len;
  int ell_state = 0, ell_k = 0;
  vtm::DevBuf d_port_loc, d_port_pos, d_twin, d_beta, d_run, d_tdesc;  // d_beta: beta d
  vtm::DevBuf d_bout, d_rho, d_kd, d_kd32;  // per port: 2 W beta / d, reflection, (g/W, d)
  vtm::DevBuf d_beta32, d_bout32;           // FP32 copies of beta d and 2 W beta / d
  vtm::DevBuf d_T64, d_T32, d_T16;         // reflection matrices (T^T blocks)
  vtm::DevBuf d_Tp32, d_Tp16;              // packed symmetric copies (symmetric plans)
  vtm::DevBuf d_Tpdf;                      // packed double-float copy (FP64 plans, kernel 12)
  vtm::DevBuf d_dfstate, d_cdf;            // kernel 12: three double-float wave slots, c
  vtm::DevBuf d_kddf;                      // (g/W, d) per port as double-float pairs (float4)
  // dataflow sweeps: tiles across the lines of each tile (CSR), per-tile done
  // counters, per-sweep tile counts and the published decision, residual
  // partials of four sweeps, waves in three slots
  vtm::DevBuf d_nbr_off, d_nbr, d_done, d_flow, d_part4, d_fstate32;
  const void* wave_slot = nullptr;  // (w_in, w_out) pairs of the sweep the last inner solve ended on
  vtm::DevBuf d_c64, d_c32;                // constant term of the sweep
  vtm::DevBuf d_state64, d_state32;        // [2][nports] (w_in, w_out) pairs
  vtm::DevBuf d_v, d_v2;                   // permuted work vectors [n]
  vtm::DevBuf d_xacc, d_r, d_bcol;         // refinement vectors [n] (global order)
  vtm::DevBuf d_partials;                  // double[max(nparts, 1024)]
  vtm::DevBuf d_ctrl;                      // SweepCtrl
  vtm::DevBuf d_hist;                      // double[history capacity]
  vtm::DevBuf d_err;                       // int error word of factor kernels
  vtm::DevBuf d_red;                       // double[2] + unsigned counter for reductions
  vtm::DevBuf d_stage_in[3], d_stage_out[3];  // device copies of host arrays, kept between calls
  int hist_cap = 0;
  vtm::SweepCtrl* h_ctrl = nullptr;        // pinned mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs0 = nullptr, evs1 = nullptr;
  // sweep-kernel autotuning and graphs, per precision
  int tuned_kernel[4] = {0, 0, 0, 0};
  int dataflow_kernel = 8;  // kernel of the last sweeps run (8 or 10 for asynchronous VTM)
  float tuned_ms[4] = {0.f, 0.f, 0.f, 0.f};
  int sweep_hint[4][8] = {};  // sweeps of refinement step i of the last solve, per precision
  int batch_hint[4][8] = {};  // the same for the batched solves
  vtm::SweepGraph sweep_graph[4];
  vtm::SweepGraph batch_graph[4];
  // per-call accounting (reset by each solve)
  int launch_count = 0;
  int sweep_launch_count = 0;
  double sweep_ms = 0.0;

  // channel form for cut entries that are not branches (controlled sources)
  // and for block Jacobi: per tile, inputs = [ports | lagged entries of its
  // rows], outputs = [ports | probes (its nodes read by lagged entries of
  // other tiles)]; the tile operator maps inputs to outputs.
  int method = VTM_METHOD_VTM;
  bool general = false;
  std::vector<int32_t> in_off, out_off;  // nparts+1
  std::vector<int32_t> in_src;           // global output feeding each input (delay 1)
  std::vector<uint8_t> in_kind;          // 0 port, 1 lagged entry
  std::vector<int32_t> in_twin;          // port input: twin's global input, else -1
  std::vector<int32_t> in_own_out;       // port input: own global output, else -1
  std::vector<int32_t> in_loc;           // local position of the input's row node
  std::vector<int32_t> in_item;          // port id or lagged-entry id
  std::vector<int32_t> res_perm;         // per tile: local input ids sorted by row node
  std::vector<uint8_t> res_run;          // run length at each run start of res_perm, else 0
  std::vector<int32_t> out_loc;          // local position of each output's node
  std::vector<int32_t> out_item;         // port id of a port output, -1 for a probe
  std::vector<int32_t> E_ld;
  std::vector<int64_t> E_off;
  int64_t E_elems = 0;
  int32_t max_in = 0, max_out = 0;
  int64_t n_in = 0, n_out = 0;
  vtm::DevBuf d_in_off, d_out_off, d_in_src, d_in_kind, d_in_twin, d_in_own_out, d_in_loc,
      d_res_perm, d_res_run, d_out_loc, d_in_coef, d_in_sigma, d_out_scale, d_out_diag, d_E_off,
      d_E_ld, d_E, d_cg, d_gin, d_gout, d_in_tile, d_in_d;

  // batched right-hand sides (batch.cu)
  std::vector<int32_t> item_tile, item_m0;
  vtm::DevBuf d_item_tile, d_item_m0, d_item_order, d_bV, d_bV32, d_bV32b, d_bstate, d_bc, d_bpart, d_btol2,
      d_bctrl, d_bres;
  bool bres_init = false;
  vtm::DevBuf d_bres2;  // the double-float residual's partials | out[128] | counter
  bool bres2_init = false;
  int batch_tuned[4] = {0, 0, 0, 0};  // batched sweep variant + 1, per precision
  int batch_tuned_R[4] = {0, 0, 0, 0};  // right-hand sides it was tuned for
  int batch_used = 0;                   // batched sweep variant + 1 of the last batched solve
  int batch_grid[32] = {0};          // grid per (precision, variant)
  // tcgen05 batched sweep: work items (tile, first row, M tiles, input
  // chunks), their offsets into the tiled BF16 copy of T_P, longest first
  int tc_nitems = 0;
  vtm::DevBuf d_tc_items, d_tc_off, d_tc_order, d_Ttc;
  // blocked batched band solves: per tile the window width W, the offset of
  // its G blocks, tiles longest first, (tile, block) list, G_f and G_b
  // (built at the first FP32 batched solve after each factorisation)
  bool bk_ready = false;
  // double-float residuals of the low-precision batched solves: A's values as
  // (h, l) pairs (state 0 not built, 1 built, 2 values out of range), the
  // scaled b, residual and iterate, per-column exponents
  int vals_df_state = 0;
  vtm::DevBuf d_vals_df, d_bdf, d_xdf, d_bexp;
  vtm::DevBuf d_bk_W, d_bk_goff, d_bk_order, d_bk_blk, d_bk_Gf, d_bk_Gb;

  // adjoint of an unsymmetric system
  vtm_plan_s* transposed = nullptr;

  std::vector<vtm::DevBuf*> all_bufs();
};

namespace vtm {

vtm_status dev_alloc(DevBuf& b, size_t bytes);
void dev_free(DevBuf& b);
template <class T>
vtm_status upload(DevBuf& b, const std::vector<T>& h, cudaStream_t s) {
  VTM_TRY(dev_alloc(b, h.size() * sizeof(T) > 0 ? h.size() * sizeof(T) : 16));
  if (!h.empty()) VTM_CUDA_TRY(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return VTM_OK;
}

bool is_device_ptr(const void* p);

// plan.cu
vtm_status assemble_local(vtm_plan_s* P);  // host band values of K_P + port tables -> device

// general.cu (channel form: lagged couplings and block Jacobi)
vtm_status build_general_operators(vtm_plan_s* P);
vtm_status general_const(vtm_plan_s* P, const double* x0_perm);
vtm_status general_sweeps(vtm_plan_s* P, double bnorm2, double target2, int budget, double* hist,
                          int hist_len, int* sweep_out, int* flag_out);
vtm_status general_inject(vtm_plan_s* P, int sweep, double* v);

// factor.cu
vtm_status factor_tiles(vtm_plan_s* P);
vtm_status build_reflections(vtm_plan_s* P);

// solve.cu
vtm_status solve_columns(vtm_plan_s* P, const double* d_b, double* d_x, int64_t nrhs, double tol,
                         vtm_info* info);
vtm_status residual_norms(vtm_plan_s* P, const double* d_x, const double* d_b, int64_t nrhs,
                          double* rel);

vtm_status residual_pair(vtm_plan_s* P, const double* x, const double* b, double* r, double* rr,
                         double* bb, float* v1 = nullptr, float* v2 = nullptr);
vtm_status solve_batched(vtm_plan_s* P, const double* d_b, double* d_x, int R, double tol,
                         vtm_info* info, bool record_hist = false);
vtm_status ensure_vals_df(vtm_plan_s* P);
int launch_residual(const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                    const double* b, int64_t n, double* partials, unsigned* counter, double* out,
                    int max_grid, cudaStream_t s);

// Launch helpers exported between translation units.
void launch_band_solve(vtm_plan_s* P, double* v, int ncols, int64_t vec_stride, cudaStream_t s);
void launch_band_solve32(vtm_plan_s* P, float* v, int ncols, int64_t vec_stride, cudaStream_t s);

}  // namespace vtm
