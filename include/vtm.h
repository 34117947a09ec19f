/*
 * vtm.h -- C ABI of libvtm, a GB300 (sm_103a) implementation of the Virtual
 * Transmission Method (VTM) of Wei & Yang, "Transmission Line Inspires A New
 * Distributed Algorithm to Solve the Linear System of Circuit",
 * arXiv 0910.0663.
 *
 * The library solves the nodal system A x = b of a circuit (Sec. II, Eq. 1).
 * A is torn into sub-circuits along virtual lossless transmission lines of
 * characteristic impedance Zc (wire tearing, Sec. V; transmission delay
 * equations, Eq. 3-5, W = 1/Zc).  Every VTM sweep (Sec. VI, Eq. 11 / Eq. 14)
 * lets each sub-circuit solve its own system loaded by W at its torn ports
 * with the incident waves on the right-hand side; the outgoing waves then
 * cross every line with one sweep of delay, and a residual norm decides
 * convergence.
 *
 * Tearing of a disjoint node partition: every branch between nodes of two
 * different parts is torn at its midpoint (two 2g conductances in series,
 * the midpoint split into twin nodes, Sec. V Steps 1-4).  Inside the library
 * each sub-circuit P is condensed onto its ports through its voltage
 * reflection matrix T_P = (W - S_P)(W + S_P)^-1 (Sec. VIII), so that a sweep
 * is w_out = T_P w_in + c_P per sub-circuit followed by the exchange
 * w_in(s) <- w_out(twin(s)).
 *
 * Conventions for every entry point:
 *  - Array arguments may live in device memory or in host memory (pageable
 *    or pinned); the library inspects each pointer.  Host arrays are copied
 *    in and out on the plan's stream.  The caller keeps ownership.
 *  - Matrices are CSR with int64 row pointers, int32 column indices sorted
 *    within each row, and float64 values.  Vectors of several right-hand
 *    sides are n x nrhs column-major (column r starts at r*n).
 *  - All device work of a plan runs on the CUDA stream given to vtm_plan
 *    (NULL = the legacy default stream).  Calls on one plan must not
 *    overlap; distinct plans are independent.
 *  - Errors are returned as vtm_status; nothing aborts the process and there
 *    is no CPU fallback.  vtm_strerror gives a message; vtm_last_error_detail
 *    gives the last detailed message of the calling thread.
 */
#ifndef VTM_H
#define VTM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vtm_plan_s* vtm_plan_t;

typedef enum {
  VTM_OK = 0,
  VTM_EINVAL = -1,       /* bad argument: size, range, empty part, pattern change */
  VTM_ENOMEM = -2,       /* device or host allocation failed */
  VTM_ESINGULAR = -3,    /* non-positive (Cholesky) or zero (LU) pivot in a local factor */
  VTM_ENOCONV = -4,      /* tolerance not met within max_sweeps / max_outer; x = last iterate */
  VTM_EDIVERGED = -5,    /* NaN/Inf or residual growth > 1e6 x initial; x = last iterate */
  VTM_ETIMEOUT = -6,     /* a bounded device-side wait ran out (persistent kernels) */
  VTM_ECUDA = -7,        /* a CUDA runtime call failed */
  VTM_EINTERNAL = -8,    /* an internal consistency check failed */
  VTM_ENOTFACTORED = -9  /* vtm_solve/vtm_adjoint before vtm_factor (or after vtm_set_values) */
} vtm_status;

/* Arithmetic of the sub-circuit applies (the reflection-matrix products). */
enum {
  VTM_PREC_FP64 = 0, /* plain FP64 VTM */
  VTM_PREC_FP32 = 1, /* FP32 T_P and waves, FP32 accumulate, inside FP64 iterative refinement */
  VTM_PREC_BF16 = 2, /* BF16 T_P, FP32 waves and accumulate, inside FP64 iterative refinement */
  VTM_PREC_FP16 = 3  /* FP16 T_P, FP32 waves and accumulate, inside FP64 iterative refinement:
                        the bytes of BF16 with a 10-bit mantissa; T_P of a symmetric plan has
                        its spectrum in (-1, 1] (Sec. VIII), so no entry leaves FP16's range */
};

/* Iteration run by a plan. */
enum {
  VTM_METHOD_VTM = 0, /* virtual transmission lines on the torn branches (Sec. VI) */
  VTM_METHOD_BJ = 1,  /* block Jacobi over the same sub-circuits (the comparison method of
                         Sec. X): every cut entry is applied with one sweep of delay */
  VTM_METHOD_ASYNC = 2 /* asynchronous VTM (Sec. XI: lines with different, varying delays):
                         one cooperative launch in which every tile reads the waves its
                         neighbours last wrote, without waiting for them (kept within eight
                         sweeps of the last residual decision; two on the older dataflow
                         kernel used where one warp per tile does not fit).  Same fixed point, timing-dependent
                         iterates.  Needs FP32/BF16/FP16 sweeps of a symmetric plan with at most
                         256 ports per sub-circuit (VTM_EINVAL at vtm_solve otherwise) */
};

typedef struct {
  int precision;     /* VTM_PREC_*; default VTM_PREC_FP64 */
  int max_sweeps;    /* sweeps per vtm_solve call, all refinement steps together; default 200000 */
  int check_every;   /* sweeps launched between two host polls of the convergence flag; default 32.
                        An inner solve (single-column or batched) first launches the sweeps
                        the same refinement step took in the plan's previous solve and the
                        launch that decides the last of them (with graphs: in groups of
                        check_every, then of check_every / 4), then polls (launches past
                        convergence return at once) */
  double inner_tol;  /* relative tolerance of each inner solve in the refinement modes;
                        0 -> 1e-5 (FP32) / 1e-3 (FP16) / 3e-3 (BF16).  An inner solve that can finish
                        the job (inner_tol x its right-hand side <= 4 tol ||b||) aims at
                        tol/2 instead.  An inner solve also ends when its residual has
                        not dropped by 10% within 64 sweeps (its rounding floor); the
                        FP64 refinement then continues. */
  int max_outer;     /* refinement steps in the FP32/BF16/FP16 modes; default 40.  Every
                        step must cut ||b - A x|| by 10x (FP32 sweeps) or 2x (BF16/FP16),
                        or by 10% once ||r|| is within that factor of the target; a step
                        that gains less ends the solve with VTM_ENOCONV (refinement
                        stalled; x = the iterate so far) */
  int method;        /* VTM_METHOD_VTM (default), VTM_METHOD_BJ (chosen at vtm_plan only) or
                        VTM_METHOD_ASYNC (switchable with VTM by vtm_set_opts) */
  int batch;         /* several right-hand sides: 0 (default) one batched iteration over
                        up to 64 columns at a time; 1: one column after the other */
  int batch_solve;   /* batched FP32 band solves: 0 (default) blocked when every half
                        bandwidth is at most 128, else row window; 1: whole column block
                        in shared memory; 2: row window in shared memory; 3: blocked --
                        rows in blocks of 64, each block one product with the inverted
                        diagonal block of the factor and its coupling to the previous
                        rows (matrices formed in FP64 at the first FP32 batched solve
                        after each factorisation, stored in FP32; VTM_EINVAL for a half
                        bandwidth above 128) */
  int l2_persist;    /* 1: during FP32/16-bit sweeps, mark the reflection matrices persisting
                        in L2 (access-policy window on the plan's stream; the context's
                        persisting carve-out is set and restored around each inner solve;
                        needs a non-default stream); 0 (default): off -- on the 2048^2
                        power grid the window saved nothing and its set-up and reset cost
                        2-3% of a solve */
  int sweep_kernel;  /* 0 (default): autotuned -- the first solve of each precision times
                        every sweep kernel that fits the plan's sub-circuits and keeps the
                        fastest; 1: direct-load kernel; 2: bulk-copy staged kernel;
                        3: 16-byte vector-load kernel, 256 threads per tile;
                        4: the same with 128 threads (p <= 128 VEC);
                        5, 6: packed symmetric kernel, 128 threads per tile, up to 85 / 64
                        registers (6 / 8 CTAs per SM) --
                        FP32/BF16/FP16 plans of a symmetric A whose sub-circuits have at
                        most 256 ports keep only the 16x16 blocks of T_P on and above
                        the diagonal (T_P is symmetric for scalar W, Sec. VIII), about
                        half the bytes per sweep; 7: the same blocks, each tile brought
                        into shared memory by one bulk copy; 8: the same blocks in one
                        cooperative launch per inner solve, each tile starting sweep k
                        once the tiles across its lines have finished sweep k - 1 (no
                        kernel boundary per sweep; same iterates as 5); 9: the same
                        blocks with one warp per tile (one CTA per SM holding
                        ceil(sub-circuits / SMs) tile warps, blocks column by column;
                        the same iteration as 5 up to rounding); 10: kernel 9's tiles
                        in one cooperative launch per inner solve (same iterates as
                        9); 11: kernel 9 with each block's products on the tensor
                        cores (warp MMAs, FP32 accumulate; the incident waves enter
                        as 16-bit hi + lo pairs scaled per tile by a power of two),
                        BF16/FP16 plans with at most 128 ports per sub-circuit;
                        12: FP64 plans of a symmetric A with at most 128 ports per
                        sub-circuit: kernel 9's organisation on the packed blocks kept
                        as hi + lo FP32 pairs (FP64 bytes, about 48 bits), waves and c
                        as such pairs, every product and sum in double-float
                        arithmetic on the FP32 pipes (GB300 runs FP64 arithmetic at a
                        small fraction of its FP32 rate); where a packed kernel does
                        not fit, 5-12 fall back to kernel 1 */
  int graphs;        /* 0 (default): replay batches of check_every sweep launches from a
                        CUDA graph when the plan has its own stream; 1: plain launches */
  int pdl;           /* 0 (default): the packed sweeps (kernels 5-7) are launched as
                        programmatic dependents of the sweep before them, so each tile
                        loads its reflection blocks and port data while the previous
                        sweep finishes, and reads the waves only once it has; 1: off */
  double* history;   /* optional host array: relative (interface) residual after each
                        sweep k=1..history_len of the first column; NULL = not recorded */
  int history_len;
  int batch_kernel;  /* batched sweep of several right-hand sides: 0 (default) autotuned
                        at the first batched solve of each precision; 1: CUDA cores,
                        persistent grid over the work list; 2: BF16 tensor cores
                        (warp MMAs, FP32 accumulate), persistent; 3, 4: the same with
                        one work item per CTA; 5: BF16 tcgen05 (128 x 64 tiles of
                        T_P streamed by bulk copies into a shared-memory ring,
                        incident waves gathered into the B operand, FP32
                        accumulators in TMEM).  A tensor-core request in another
                        precision, or (2, 4) with a column count that is not a
                        multiple of 8, runs the CUDA-core variant */
  int wait_polls;    /* polls a bounded device-side wait of the dataflow sweeps
                        (kernels 8 and 10) makes before it gives up with VTM_ETIMEOUT;
                        0: default 4194304 (a few seconds).  The bulk-copy waits of
                        kernels 2 and 7 keep their own limit: a CTA never leaves while a
                        copy into its shared memory is in flight */
  int flow_lag;      /* 0 (default): a dataflow tile starts sweep k once the residual
                        decision of sweep k - 2 is out.  -1: every tile waits for the
                        decision of its own sweep, which cannot come -- a host-made hang
                        that the bounded waits end with VTM_ETIMEOUT (a test of that
                        path; the plan stays usable) */
  int band_solve;    /* single-column FP32 band solves of half bandwidth <= 32 (the
                        right-hand-side preparation and recovery of low-precision
                        solves): 0 (default) factor columns streamed by bulk copies
                        through a shared-memory ring per tile; 1: the same arithmetic
                        with register prefetch.  Both give the same bits */
} vtm_opts;

typedef struct {
  int sweeps;        /* total sweeps run (all refinement steps) */
  int outer_steps;   /* refinement steps (1 in FP64 mode) */
  double relres;     /* max over columns of ||b - A x||_2 / ||b||_2, from an FP64 SpMV of the returned x */
  double t_solve_ms; /* device time of the call (CUDA events on the plan's stream) */
  int first_sweep_converged; /* sweep k at which the interface residual first met tol (FP64 mode) */
  int kernel_launches;       /* kernels libvtm launched during the call */
  int sweep_launches;        /* sweep-kernel launches (including launches that found the
                                convergence flag already set and returned at once) */
  double t_sweeps_ms;        /* device time of the sweep-kernel launches (CUDA events around
                                each batch of back-to-back launches on the plan's stream) */
} vtm_info;

typedef struct {
  int64_t n;
  int32_t nparts;
  int64_t nports;        /* two per torn branch */
  int64_t nlagged;       /* cut entries that are not branches (controlled sources) */
  int64_t sum_p2;        /* sum over sub-circuits of p_P^2 (reflection-matrix entries) */
  int32_t max_ports;     /* largest p_P */
  int32_t max_nodes;     /* largest sub-circuit */
  int32_t max_band;      /* largest half-bandwidth of a local matrix after reordering */
  int32_t symmetric;     /* 1: A symmetric -> Cholesky; 0: LU without pivoting */
  int64_t t_bytes;       /* bytes of the stored reflection matrices (all precisions kept) */
  int64_t factor_bytes;  /* bytes of the stored local factors */
  int32_t sweep_kernel;  /* sweep kernel in use for the plan's precision (see vtm_opts) */
  int64_t sum_tri;       /* sum over sub-circuits of p_P (p_P + 1) / 2: the entries of the
                            symmetric reflection matrices on and above the diagonal */
  int64_t packed_bytes;  /* bytes of the packed symmetric copies (0 if none) */
  int32_t batch_kernel;  /* batched sweep variant of the last batched solve (see
                            vtm_opts.batch_kernel; 0: none yet) */
} vtm_plan_stats;

/* vtm_plan -- wire tearing (Sec. V) and the port table.
 * n: unknowns.  rowptr[n+1], colidx[nnz], vals[nnz]: A in CSR (host or device).
 * partition[n]: sub-circuit of each node, values in [0, nparts); every part
 * must be non-empty.  Zc > 0: characteristic impedance of every virtual line
 * (W = 1/Zc, the choice W = alpha I of Sec. VIII).  opts may be NULL.
 * stream: a cudaStream_t (or NULL).  On success *out owns all device buffers.
 * Errors: VTM_EINVAL (n <= 0, nparts <= 0, partition out of range, empty
 * part, Zc <= 0 or not finite, unsorted or out-of-range column indices),
 * VTM_ENOMEM, VTM_ECUDA. */
vtm_status vtm_plan(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                    const int32_t* partition, int32_t nparts, double Zc, const vtm_opts* opts,
                    void* stream, vtm_plan_t* out);

/* vtm_set_values -- new values for the same sparsity pattern (gradients,
 * finite differences).  The set of torn branches (cut pairs with a positive
 * symmetric conductance) must not change: VTM_EINVAL otherwise.  The plan
 * must be factored again before the next solve. */
vtm_status vtm_set_values(vtm_plan_t plan, const double* vals);

/* Characteristic admittance of the virtual lines (Sec. VIII: the speed of
 * convergence depends on W; the paper lists five choices).  Under midpoint
 * tearing C_P = diag(2 g_s) is diagonal, so every choice is one value per
 * line, shared by its two ports. */
enum {
  VTM_W_ALPHA = 0, /* W = alpha I (choice 1); the plan's default is alpha = 1/Zc */
  VTM_W_DIAG = 1,  /* W = diag(C) = 2 g_e on line e (choice 2; also choice 3, W = C);
                      the VTM iteration then equals block Jacobi sweep by sweep */
  VTM_W_WOB = 2,   /* W = alpha C = alpha 2 g_e (choice 4, weighted overlapped block) */
  VTM_W_SCA = 3,   /* diagonal of the partial input admittance C - E~ D~^-1 F~ with D~ the
                      rows of the sub-circuit within `radius` branches of the port's node
                      (choice 5, small elements dropped to the pattern of C); a line takes
                      the value of its end in the lower-numbered sub-circuit */
  VTM_W_LINE = 4   /* one value per port, given by the caller */
};

/* vtm_set_admittance -- choose the line admittances (see the enum above).
 * alpha: used by VTM_W_ALPHA and VTM_W_WOB, > 0.  radius: VTM_W_SCA, 0..8
 * (the dense partial solve of a port is limited to 512 nodes).  W: VTM_W_LINE
 * only, nports values in the port order of vtm_get_ports (host or device),
 * positive and equal at both ports of a line.  DIAG, WOB and SCA follow the
 * values: vtm_set_values recomputes them.  With any choice other than
 * VTM_W_ALPHA the library carries power waves w / sqrt(W_s), under which the
 * condensed operator of a symmetric A stays symmetric.  The plan must be
 * factored again.  VTM_EINVAL (choice unchanged) for an unknown kind or a bad
 * alpha, radius or W; VTM_ESINGULAR if a partial sub-circuit matrix is
 * singular. */
vtm_status vtm_set_admittance(vtm_plan_t plan, int kind, double alpha, int radius, const double* W);

/* vtm_get_admittance -- the line admittance of every port (nports doubles,
 * port order of vtm_get_ports; host or device). */
vtm_status vtm_get_admittance(vtm_plan_t plan, double* W);

/* vtm_set_opts -- replace the options of a plan (precision, limits, history).
 * VTM_EINVAL for a precision outside 0..3, a negative history_len, a history
 * length without an array, a sweep_kernel outside 0..12, a batch_kernel
 * outside 0..5, a negative wait_polls or a flow_lag other than 0 and -1; the
 * plan keeps its previous options then. */
vtm_status vtm_set_opts(vtm_plan_t plan, const vtm_opts* opts);

/* vtm_factor -- per sub-circuit factorisation of the condensed local matrix
 * K_P = A_PP + sum_s (g_s - 4 g_s^2/(2 g_s + W)) e_l(s) e_l(s)^T (the matrix
 * of Eq. 11 after eliminating the twin rows) by banded Cholesky (symmetric A)
 * or banded LU without pivoting, in FP64; then the reflection matrices
 * T_P = (W - S_P)(W + S_P)^-1 (Sec. VIII) from p_P banded solves each, kept
 * in FP64 and in the precision selected by opts.  Errors: VTM_ESINGULAR. */
vtm_status vtm_factor(vtm_plan_t plan);

/* vtm_solve -- solve A x = b by VTM sweeps (Sec. VI, Eq. 11/14) with zero
 * initial waves, until ||b - A x||_2 <= tol ||b||_2 for every column.
 * b, x: n x nrhs column-major, host or device; x is output only.  tol > 0.
 * Host arrays are copied through device buffers the plan keeps between calls
 * (grown when a call needs more; freed by vtm_destroy), pinned host memory at
 * the link's rate.
 * The convergence test after every sweep uses the residual of the torn
 * branches (the interior rows of each sub-circuit are solved exactly); the
 * returned info->relres comes from an FP64 SpMV of the returned x.
 * Errors: VTM_ENOTFACTORED, VTM_EINVAL, VTM_ENOCONV, VTM_EDIVERGED (x then
 * holds the last iterate and info is filled). */
vtm_status vtm_solve(vtm_plan_t plan, const double* b, double* x, int64_t nrhs, double tol,
                     vtm_info* info);

/* vtm_adjoint -- solve A^T lam = g (same tearing; for a symmetric A the same
 * operators, otherwise a transposed plan built and factored on first use).
 * Arguments as vtm_solve. */
vtm_status vtm_adjoint(vtm_plan_t plan, const double* g, double* lam, int64_t nrhs, double tol,
                       vtm_info* info);

/* vtm_plan_get_stats -- sizes of the tearing and of the stored operators. */
vtm_status vtm_plan_get_stats(vtm_plan_t plan, vtm_plan_stats* stats);

/* vtm_get_ports -- the port table (host arrays of length stats.nports):
 * node = the port's node, remote = the node across the torn branch,
 * part = owning sub-circuit, twin = the port at the other end of the line.
 * Ports are grouped by sub-circuit, then ordered by (node, remote).
 * Any pointer may be NULL. */
vtm_status vtm_get_ports(vtm_plan_t plan, int32_t* node, int32_t* remote, int32_t* part,
                         int32_t* twin);

/* vtm_get_reflection -- copy T_P of sub-circuit `part` (p_P x p_P, row-major,
 * FP64, ports in vtm_get_ports order) into host array T (capacity `cap`
 * doubles); *p receives p_P.  Requires vtm_factor. */
vtm_status vtm_get_reflection(vtm_plan_t plan, int32_t part, double* T, int64_t cap, int32_t* p);

/* vtm_get_reflection_stored -- T_P of sub-circuit `part` as the sweeps of the
 * plan's precision read it, converted to FP64: for FP32/BF16/FP16 plans the
 * packed 16x16 blocks on and above the diagonal (symmetric plans with at most
 * 256 ports per sub-circuit; each stored entry is the rounded mean of T_P(s,q)
 * and T_P(q,s), Sec. VIII symmetry) or else the full low-precision copy; for
 * FP64 plans the FP64 matrix.  Layout, port order and wave scaling as
 * vtm_get_reflection (p_P x p_P row-major in host array T of capacity `cap`),
 * so that T - vtm_get_reflection(T) is the storage rounding the sweeps see.
 * *stored receives the element size in bytes (8, 4 or 2) and *packed 1 if the
 * packed blocks were read.  Requires vtm_factor. */
vtm_status vtm_get_reflection_stored(vtm_plan_t plan, int32_t part, double* T, int64_t cap,
                                     int32_t* p, int32_t* stored, int32_t* packed);

/* vtm_march -- backward-Euler transient of an RC network with the plan's
 * matrix A = G + C/h: for k = 1..nsteps
 *   A x_k = p_k + (C/h) x_{k-1},
 * each step solved to tol like vtm_solve, starting from x_{k-1} (warm start:
 * the refinement's first inner problem is A d = b_k - A x_{k-1}).
 * cdiag[n]: C/h per node (the part of A's diagonal carried by the state).
 * p: n x nsteps injections (column k-1 = step k).  x0[n]: initial state, or
 * NULL for zero.  X: n x nsteps output (column k-1 = x_k).  Arrays host or
 * device.  info: sweeps and outer_steps summed over the steps, relres the
 * largest, t_solve_ms the whole march.  Errors as vtm_solve; a failing step
 * ends the march (vtm_last_error_detail names it). */
vtm_status vtm_march(vtm_plan_t plan, const double* cdiag, const double* p, const double* x0,
                     double* X, int64_t nsteps, double tol, vtm_info* info);

/* vtm_residual_norm -- rel[r] = ||b_r - A x_r||_2 / ||b_r||_2 for each of
 * nrhs columns, in FP64 on the plan's stream (A = the plan's current values).
 * x, b: n x nrhs column-major (host or device); rel: host array[nrhs]. */
vtm_status vtm_residual_norm(vtm_plan_t plan, const double* x, const double* b, int64_t nrhs,
                             double* rel);

/* ---- resistor networks: branch map and gradients (adjoint of Eq. 1) ----
 * A netmap ties a branch list (e: i -- j, conductance g_e) and node-to-ground
 * conductances to the CSR pattern of A = sum_e g_e (e_i - e_j)(e_i - e_j)^T
 * + diag(ground) (nodal analysis, Sec. II, Eq. 1; Lemma 1). */
typedef struct vtm_netmap_s* vtm_netmap_t;

/* vtm_netmap_create -- rowptr[n+1], colidx[nnz] (host or device): the CSR
 * pattern, which must hold every diagonal and both (i,j), (j,i) of every
 * branch; ei[nedges], ej[nedges] (int64, host or device): branch ends, no
 * self-loops, no parallel branches.  Work of the map runs on `stream`.
 * Errors: VTM_EINVAL. */
vtm_status vtm_netmap_create(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                             int64_t nedges, const int64_t* ei, const int64_t* ej, void* stream,
                             vtm_netmap_t* out);

/* vtm_netmap_values -- vals[nnz] = values of A for branch conductances
 * g[nedges] and ground[n] (NULL = no ground); all device arrays; each
 * diagonal is summed in a fixed order (deterministic).  Stream-ordered. */
vtm_status vtm_netmap_values(vtm_netmap_t map, const int64_t* rowptr, const double* g,
                             const double* ground, double* vals);

/* vtm_netmap_gradient -- for lam = A^-T dL/dx (vtm_adjoint) and x (n x nrhs,
 * column-major, device): grad_g[e] = -sum_r (lam_i - lam_j)(x_i - x_j) and,
 * if grad_ground is not NULL, grad_ground[i] = -sum_r lam_i x_i.  dL/db is
 * lam itself.  Device arrays; stream-ordered. */
vtm_status vtm_netmap_gradient(vtm_netmap_t map, const double* lam, const double* x, int64_t nrhs,
                               double* grad_g, double* grad_ground);

void vtm_netmap_destroy(vtm_netmap_t map);

/* vtm_residual_norm_noalloc -- the same relative residual norms as
 * vtm_residual_norm, for callers that cannot allocate device memory (a
 * simulator whose pool owns the whole device, a loop that must not call
 * cudaMalloc, code that only holds buffers lent to it).  The paper has no
 * counterpart; this is a service of the library.
 * Needs no plan and allocates nothing: rowptr[n+1], colidx[nnz], vals[nnz],
 * x and b (n x nrhs column-major) must all be device memory of the current
 * device (or managed memory); rel is a host array[nrhs].  Work runs on `stream` (a cudaStream_t or NULL) and the call
 * returns after it finished.  Scratch is a fixed 20,736-byte __device__ array
 * in the library, present on every GPU that loads it until the process
 * exits; hence nrhs <= 64 (VTM_EINVAL beyond).  The first call on a device
 * looks up that array's address with the device current; make that first
 * call before any stream capture.  All calls on a device share the array,
 * so calls that overlap on the GPU (other streams or threads) race; the
 * array keeps the last call's sums and the call clears what must start at
 * zero.  Errors: VTM_EINVAL (sizes, NULL, host pointers, memory of another
 * device; nothing is launched then), VTM_ECUDA. */
vtm_status vtm_residual_norm_noalloc(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                                     const double* vals, const double* x, const double* b,
                                     int64_t nrhs, double* rel, void* stream);

void vtm_destroy(vtm_plan_t plan);
const char* vtm_strerror(vtm_status status);
const char* vtm_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* VTM_H */
