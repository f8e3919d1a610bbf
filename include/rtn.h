/*
 * rtn.h -- C ABI of the B300-native Real-time Neural MPC hot path.
 *
 * Method: Salzmann, Kaufmann, Arrizabalaga, Pavone, Scaramuzza, Ryll,
 * "Real-time Neural MPC", RA-L 2023.  For every shooting node k of every
 * controller instance b the library
 *   (a1) evaluates the residual network f_D and its input Jacobian J_D
 *        (the first-order local model of Sec. III-A, Eq. 4),
 *   (a2) forms the RK4 discretisation phi of f_F + f_D* (Sec. II, Eq. 1;
 *        f_F is the nominal quadrotor model of Sec. V, Eq. 6) with the
 *        sensitivities A_k, B_k and the defect c_k = phi_k - x_{k+1} of the
 *        continuity condition (Eq. 2),
 *   (a3) solves the linear-quadratic subproblem of Sec. III-A with the
 *        tracking cost of Sec. V by a Riccati sweep,
 *   (a4) applies the feedback response of Sec. III-B (Fig. 2): the measured
 *        x0 enters, the iterate is updated and the first command is sent,
 *   (a5) steps a plant (nominal model + a true residual) for closed loops,
 *   (a6) trains the residual network (MSE, Adam; Sec. VI).
 *
 * Conventions (all entry points):
 *   - nx = 13: x = [p(3), q(4) w-first, v(3), omega(3)];  nu = 4: rotor thrusts.
 *   - Node-packed arrays: instance b owns N_b nodes.  States are packed as
 *     [sum_b (N_b + 1)][13] (x_0..x_N per instance, instance-major), inputs
 *     and per-node outputs as [sum_b N_b][...] in the same order.
 *   - Matrices are row-major float32: A [node][13][13], B [node][13][4],
 *     J_D [node][no][17] (columns: 13 state, then 4 input derivatives; no =
 *     the network's outputs, 3 or 6, see rtn_mlp).
 *   - Pointers documented "dev" are device pointers owned by the caller; the
 *     library never frees them.  "host" pointers are read during the call.
 *   - Every call is asynchronous on the stream given to rtn_create, except
 *     where stated.  Argument errors are returned synchronously; per-instance
 *     numerical failures are written to inst_status (dev int [B]).
 *   - No C++ exception crosses this boundary.  rtn_last_error() returns a
 *     description of the last failure on the context.
 */
#ifndef RTN_H
#define RTN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtn_ctx rtn_ctx;

typedef enum {
  RTN_OK = 0,
  RTN_E_INVAL = 1,       /* bad argument (sizes, NULL, unsupported shape) */
  RTN_E_CUDA = 2,        /* a CUDA runtime call failed */
  RTN_E_NONFINITE = 3,   /* per instance: NaN/Inf in the measured state */
  RTN_E_NOT_PD = 4,      /* per instance: R + B'PB not positive definite */
  RTN_E_TIMEOUT = 5,     /* a bounded device wait gave up */
  RTN_E_NOMEM = 6,       /* device allocation failed */
  RTN_E_UNSUPPORTED = 7, /* feature not available for this configuration */
  RTN_E_NOT_CONVERGED = 8 /* per instance: the box-constrained QP's active sets
                             did not settle within box_max_iter subproblems;
                             the step applied is the last one clamped to the box */
} rtn_status;

/* arithmetic of the network evaluation (a1) */
enum {
  RTN_FP32 = 0,   /* FP32-accurate: tcgen05 kind::tf32 with weights and
                     activations split hi + lo in TF32 (three MMAs per
                     product), FP32 accumulation */
  RTN_BF16 = 1,   /* tcgen05, BF16 operands, FP32 accumulation, one pass */
  RTN_BF16X2 = 2, /* tcgen05, activations/tangents split hi+lo in BF16
                     (two passes), FP32 accumulation */
  RTN_FP8 = 3     /* tcgen05 kind::f8f6f4: every weight matrix quantised
                     at create to e4m3 with a per-layer scale amax/448 (the
                     context's network is then the dequantised one); the
                     hidden->hidden GEMMs forward and backward multiply the
                     e4m3 weights with activations / adjoints stored as three
                     e4m3 pieces (hi + mid + lo, ~12 significant bits) in
                     three MMAs with FP32 accumulation; the input layer, the
                     folded first backward layer and the Jacobian GEMM as in
                     RTN_BF16X2.  Layered reverse mode only: tile mode 6
                     by default, mode 7 (the hidden GEMMs on CTA pairs)
                     selectable where the padded width is a multiple of 256;
                     3-output networks with at least one hidden->hidden
                     layer */
};

/* plant residual used by rtn_plant_step / rtn_closed_loop */
enum { RTN_PLANT_NOMINAL = 0, RTN_PLANT_DRAG = 1, RTN_PLANT_MLP = 2 };

/* Residual network: n_layers weight matrices (hidden tanh layers then one
 * linear output layer).  widths has n_layers+1 entries, widths[0] = 17,
 * widths[n_layers] = no, the outputs:
 *   no = 3: a world-frame linear acceleration residual added to dv/dt;
 *   no = 6: the full residual of Eq. 7, [0; 0; f_theta; f_psi]: rows 0-2
 *     the linear acceleration (added to dv/dt), rows 3-5 the body angular
 *     acceleration (added to domega/dt).  Two separate networks theta, psi
 *     are one 6-output network whose first layer stacks their rows and whose
 *     deeper layers are block-diagonal.  The 6-output residual runs on the
 *     FP32 path (RTN_FP32; first or second order).
 * W[l] is host float32 row-major [widths[l+1]][widths[l]], b[l] host float32
 * [widths[l+1]].  Copied at rtn_create; the caller keeps ownership. */
typedef struct {
  int n_layers;
  const int* widths;
  const float* const* W;
  const float* const* b;
} rtn_mlp;

/* Quadrotor parameters (Sec. V): mass [kg], diagonal inertia [kg m^2],
 * arm length [m] (X layout of Fig. 3), yaw-torque coefficient, maximum
 * thrust per rotor [N], gravity [m/s^2]. */
typedef struct {
  double mass, Jx, Jy, Jz, arm, c_tau, u_max, g;
} rtn_quad;

typedef struct {
  int precision;    /* RTN_FP32 / RTN_BF16 / RTN_BF16X2 / RTN_FP8 */
  int riccati_f64;  /* Riccati sweep arithmetic: 0 FP32 (the Cholesky of
                       R + B'PB in FP32); 1 FP64 throughout; 2 FP32 with the
                       Cholesky of R + B'PB in FP64 (R + B'PB formed in FP32,
                       its factor rounded to FP32 for the solves of the gains
                       [K | k]) */
  int shift;        /* 1: shift the iterate by one stage after every RTI step */
  int box_qp;       /* 1: the QP carries the thrust bounds 0 <= u_k + du_k <= u_max
                       (Sec. V) and is solved by a primal-dual active-set method
                       whose subproblems are masked Riccati sweeps; 0: no bounds
                       in the QP, only the sent u_0 is clamped */
  int box_max_iter; /* subproblems per QP at most (0: 20) */
  int second_order; /* 1: linearise with the second-order local model of Eq. 4,
                       f_D* = f_D + J_D dz + 1/2 dz' H_D dz per output, H_D the
                       network Hessian at the node (forward-over-forward, FP32);
                       needs RTN_FP32, the quadrotor model and a network.  The
                       RK4 stages see the quadratic term along the state
                       deviation (u is held over the interval). 0: Eq. 4 to
                       first order (J_D only) */
  int fused_qp;     /* 1: every RTI step runs the RK4 linearisation (a2) and
                       the QP with the feedback (a3 + a4) in one persistent
                       launch: warps take RK4 work (node columns, longest
                       horizon first) from an atomic queue, then one
                       instance's QP each, which waits (bounded, ~2 s, then
                       RTN_E_TIMEOUT for that instance) until its nodes are
                       linearised; applies to the quadrotor model with a
                       3-output first-order residual, the FP32 sweep and no
                       bounds in the QP (other contexts run the separate
                       launches).  0: separate launches */
  int train_bf16;   /* GEMMs of rtn_train and rtn_mse_grad: 0 BF16 hi + lo
                       split operands (three MMAs per product, relative error
                       ~1e-5); 1 operands rounded to BF16 (one MMA per product:
                       a third of the tensor work and half the operand bytes),
                       FP32 accumulation and FP32 master weights in either */
  int qp_group;     /* threads per instance in the Riccati sweep and
                       feedback: 32 (one warp per instance), 16 (two
                       instances per warp: half the warps, twice the
                       instances in flight; faster when the batch is
                       throughput-bound or the factorisation is in FP64,
                       slower when the longest horizon's sequential chain
                       decides or with box_qp) or 256 (one block per
                       instance, each step's products spread over the block:
                       the latency of small batches, e.g. one controller;
                       not with box_qp or horizons beyond ~110 nodes, which
                       take 32 instead); 0 chooses: 32 with box_qp, else 256
                       when the batch has at most one instance per SM, else
                       16 with riccati_f64 = 2,
                       else 16 when the batch's nodes exceed the resident
                       warps of the sweep x the longest horizon, else 32.
                       The result does not depend on it */
} rtn_options;

/* Create a controller batch of `batch` instances with horizons N[b] >= 1 and
 * step sizes dt[b] > 0 (host arrays [batch]).  Q, R, Q_N are host diagonals
 * (nx, nu, nx); Q_N may be NULL (then Q_N = Q).  mlp may be NULL (nominal
 * model only).  opt may be NULL (FP32, FP32 sweep, shift on).  cuda_stream is
 * a cudaStream_t (NULL = legacy default stream).
 * Two models:
 *   nx = 13, nu = 4: the quadrotor of Sec. V (quad required); network 17 -> 3
 *     (or 17 -> 6, the full residual, with RTN_FP32; RTN_E_UNSUPPORTED with
 *     the tensor-core precisions);
 *   nx = 2, nu = 1: the double integrator of the runtime analysis (Sec. IV,
 *     Eq. 5): x = (p, v), u = commanded acceleration, f_F = (v, u); the
 *     network maps z = (p, v, u) to 1 output added to dv/dt (any hidden
 *     widths up to 65536); quad is ignored (may be NULL); opt must select
 *     RTN_FP32 without box_qp or riccati_f64 (RTN_E_UNSUPPORTED otherwise);
 *     the QP runs in FP32 and has no input bounds (u0 is sent unclamped).
 *     Every entry point below then uses nx = 2, nu = 1 in its layouts (fD
 *     [sum N_b][1], JD [sum N_b][1][3]); rtn_qp_solve, rtn_plant_step,
 *     rtn_closed_loop, the tile autotuner, tracing and the training calls
 *     return RTN_E_UNSUPPORTED.
 * The iterate starts at x_k = 0 (quadrotor: q = identity, u_k = hover;
 * double integrator: u_k = 0); see rtn_reset.  Synchronous.  Returns
 * RTN_E_INVAL on bad sizes, RTN_E_NOMEM/RTN_E_CUDA on device failures (then
 * *out is NULL). */
rtn_status rtn_create(rtn_ctx** out, int nx, int nu, int batch, const int* N, const double* dt,
                      const double* Q, const double* R, const double* Q_N, const rtn_quad* quad,
                      const rtn_mlp* mlp, const rtn_options* opt, void* cuda_stream);

/* Free every device buffer of the context (synchronises its stream). */
void rtn_destroy(rtn_ctx* ctx);

/* Description of the last error on ctx (or of the last failed rtn_create when
 * ctx is NULL).  Valid until the next call on the same context. */
const char* rtn_last_error(const rtn_ctx* ctx);

/* Sizes of the node-packed layout: total nodes sum N_b and states sum(N_b+1). */
rtn_status rtn_sizes(const rtn_ctx* ctx, int* n_nodes, int* n_states);

/* Initial iterate (Sec. III-B needs an iterate to linearise around):
 * x_k = x0[b] for every k, u_k = m g / 4 (double integrator: 0).  x0: dev
 * float [B][nx]. */
rtn_status rtn_reset(rtn_ctx* ctx, const float* x0);

/* Copy the iterate in or out: x dev float [sum(N_b+1)][13], u dev float
 * [sum N_b][4]. */
rtn_status rtn_set_iterate(rtn_ctx* ctx, const float* x, const float* u);
rtn_status rtn_get_iterate(rtn_ctx* ctx, float* x, float* u);

/* (a1) Data-driven preparation (Sec. III-B): f_D and J_D at every node of the
 * given points.  x dev [sum(N_b+1)][13] (x_N rows are ignored), u dev
 * [sum N_b][4]; outputs fD dev [sum N_b][no], JD dev [sum N_b][no][17].  Uses
 * the precision chosen at create.  RTN_E_UNSUPPORTED if the context has no
 * network. */
rtn_status rtn_mlp_eval(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD);

/* (f4) Second-order data-driven preparation (Eq. 4 to second order): f_D,
 * J_D as rtn_mlp_eval and the Hessian HD dev [sum N_b][no][17][17] (both
 * triangles, HD[n][r][i][j] = d^2 f_D,r / dz_i dz_j) at every node, in FP32.
 * RTN_E_UNSUPPORTED unless the context was created with second_order. */
rtn_status rtn_mlp_hess(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD, float* HD);

/* (a1)+(a2) Linearise every node (Eq. 2 with the local model of Eq. 4):
 * fD, JD as above (may be NULL), A dev [sum N_b][13][13], B dev
 * [sum N_b][13][4], c dev [sum N_b][13] = phi(x_k, u_k) - x_{k+1}. */
rtn_status rtn_linearize(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD,
                         float* A, float* B, float* c);

/* (a3)+(a4) Solve the QP of Sec. III-A for given A, B, c around the points
 * x, u (layouts as above) with references xref dev [sum(N_b+1)][13], uref dev
 * [sum N_b][4] and measured states x0 dev [B][13].  Writes the step
 * dx dev [sum(N_b+1)][13], du dev [sum N_b][4] and inst_status dev int [B]
 * (RTN_OK, RTN_E_NOT_PD, RTN_E_NONFINITE; failed instances get a zero step;
 * with box_qp also RTN_E_NOT_CONVERGED, see rtn_options). */
rtn_status rtn_qp_solve(rtn_ctx* ctx, const float* A, const float* B, const float* c,
                        const float* x, const float* u, const float* xref, const float* uref,
                        const float* x0, float* dx, float* du, int* inst_status);

/* One real-time iteration (Sec. III-B) on the context's iterate: a1..a4,
 * then the iterate update (w += dw), the sent command u0 = clamp(u_0, 0,
 * u_max) and (option) the shift.  x0 dev [B][13] (measured states), xref,
 * uref as in rtn_qp_solve, u0_out dev [B][4], inst_status dev int [B] (may be
 * NULL).  Failed instances keep their iterate and send uref's first entry. */
rtn_status rtn_rti_step(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref,
                        float* u0_out, int* inst_status);

/* rtn_rti_step with HOST buffers (Sec. III-B): x0 host [B][13], xref host
 * [sum(N_b+1)][13], uref host [sum N_b][4] in, u0_out host [B][4] and
 * inst_status host int [B] (may be NULL) out.  The inputs are read only by
 * the QP, so they are copied to device buffers owned by the context on a
 * second stream while the network pass and RK4 run on the context's stream;
 * the QP waits for the copies, u0 and the status are copied back on the
 * context's stream.  Asynchronous like the other calls: the host inputs
 * must stay unchanged and the outputs are valid only after the context's
 * stream has been synchronised.  Page-locked host memory lets the copies
 * overlap; pageable memory gives the same results with the copies staged
 * by the driver.  RTN_E_UNSUPPORTED for the double-integrator model. */
rtn_status rtn_rti_step_host(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref,
                             float* u0_out, int* inst_status);

/* Subproblems (masked Riccati sweeps) each instance's last box-constrained QP
 * needed: host int [B] (1 = the unconstrained solution was feasible).
 * Synchronous.  RTN_E_UNSUPPORTED unless the context was created with box_qp. */
rtn_status rtn_box_iterations(rtn_ctx* ctx, int* iters);

/* (a5) Plant step for every instance: nsub RK4 sub-steps of dt_b/nsub of the
 * true dynamics f_F + residual (kind RTN_PLANT_*), then q <- q/|q|, all in
 * FP64.  x dev double [B][13] in, u dev float [B][4], x_next dev double
 * [B][13] (may alias x).  RTN_PLANT_MLP uses the context's network in FP64
 * and needs widths <= 64. */
rtn_status rtn_plant_step(rtn_ctx* ctx, int kind, const double* x, const float* u, double* x_next,
                          int nsub);

/* Closed loop of `steps` control steps, captured once as a CUDA graph and
 * replayed: RTI step from the plant state, plant step with u0 (4 RK4
 * sub-steps), record.  xref_traj dev float [B][T][13] and uref_traj dev float
 * [B][T-1][4] are sampled on each instance's dt grid with
 * T >= steps + max N_b + 1; step t uses rows t..t+N_b.  x_plant dev double
 * [B][13] holds the initial plant state and receives the final one.
 * traj_out dev float [steps][B][13] (may be NULL) receives the plant state
 * after every step, u_out dev float [steps][B][4] (may be NULL) the sent
 * commands.  The iterate is NOT reset: call rtn_reset first.  Synchronous. */
rtn_status rtn_closed_loop(rtn_ctx* ctx, int steps, int plant_kind, const float* xref_traj,
                           const float* uref_traj, int T, double* x_plant, float* traj_out,
                           float* u_out);

/* (a6) Ground-truth residual targets of the drag simulator for training:
 * Y[s] = -R(q) diag(0.3, 0.3, 0.1) R(q)' v - 0.01 |v| v  (world-frame
 * acceleration), X dev [n][13], Y dev [n][3], FP32. */
rtn_status rtn_drag_targets(rtn_ctx* ctx, const float* X, int n, float* Y);

/* (a6) Mean-squared-error loss 1/(no n) sum |f_D(x, u) - y|^2 of the context's
 * network on n samples (X dev [n][13], U dev [n][4], Y dev [n][no]) and its
 * gradient: grad dev float [n_weights + n_biases] packed as all W[l]
 * (row-major, layer order) then all b[l]; loss dev float [1].  The GEMMs of
 * rtn_train (split BF16 operands, FP32 accumulation: relative error ~1e-5;
 * with rtn_options.train_bf16 BF16 operands, ~1e-2) and FP32 elementwise
 * steps. */
rtn_status rtn_mse_grad(rtn_ctx* ctx, const float* X, const float* U, const float* Y, int n,
                        float* grad, float* loss);

/* (a6) Train the context's network in place (Sec. VI: MSE, Adam with
 * b1 = 0.9, b2 = 0.999, eps = 1e-8, bias correction): `epochs` passes over
 * the n samples in consecutive minibatches of `batch` (the remainder of each
 * pass is skipped), learning rate lr.  FP32 master weights; the forward,
 * backward and weight-gradient GEMMs run on the tcgen05 tensor cores with
 * BF16 hi + lo split operands (three MMAs per product; with
 * rtn_options.train_bf16 BF16 operands, one MMA) and FP32 accumulation,
 * their bias / tanh / tanh' epilogues fused; one fused Adam launch per step
 * for every weight matrix (which also refreshes the split weights) and the
 * biases.  Adam state persists across calls.  loss_out (host, may be
 * NULL) receives the loss of every step [epochs * (n / batch)].  Afterwards
 * the network copies of the inference kernels and of the plant are
 * refreshed.  Synchronous. */
rtn_status rtn_train(rtn_ctx* ctx, const float* X, const float* U, const float* Y, int n,
                     int epochs, int batch, float lr, float* loss_out);

/* Current FP32 parameters to host memory, packed as in rtn_mse_grad. */
rtn_status rtn_get_params(rtn_ctx* ctx, float* W, float* b);

/* Tile shapes of the tensor-core network kernel (the autotuner's search
 * space).  rtn_tc_variants: number of compiled shapes.  rtn_tc_variant_info:
 * nodes per CTA (per CTA pair in mode 5; 0 in modes 6, 7), operand mode
 * in *split (0 single BF16; 1, 2 split hi + lo on one CTA; 3 is not used;
 * 4 split, reverse mode: values forward, three output
 * adjoints backward; 5 the same on CTA pairs; 6 split, reverse mode layered:
 * one GEMM per layer over all nodes, 2 L launches, its buffers allocated
 * when the shape is first selected; 7 as 6 with the hidden forward and
 * backward GEMMs on CTA pairs, hidden width a multiple of 256) and pipeline
 * depth of shape idx,
 * *fits = 1 if it can run this context's network and precision.  rtn_tc_select: use shape idx
 * (RTN_E_UNSUPPORTED if it does not fit).  rtn_autotune: time every fitting
 * shape on the context's current iterate (synchronous; 1 warm-up + 3 timed
 * calls each), keep the fastest, return its index and time per call [ms].
 * Only for contexts created with RTN_BF16 / RTN_BF16X2 / RTN_FP8 (FP8: the
 * layered shapes, tile modes 6 and 7, only). */
rtn_status rtn_tc_variants(rtn_ctx* ctx, int* count);
rtn_status rtn_tc_variant_info(rtn_ctx* ctx, int idx, int* npc, int* split, int* stages,
                               int* fits);
rtn_status rtn_tc_select(rtn_ctx* ctx, int idx);
rtn_status rtn_autotune(rtn_ctx* ctx, int* best_idx, float* best_ms);

/* Phase tracing of the fused tensor-core kernels (profiling aid, compiled in
 * only when the library is built with -DRTN_TRACE=1; otherwise enable != 0
 * returns RTN_E_UNSUPPORTED).  enable != 0
 * makes every later network evaluation record %globaltimer stamps [ns] of
 * CTA 0 into a device buffer of RTN_TC_TRACE_LEN entries: entry
 * ((i * (L + 1) + l) * 8 + f) for the i-th tile of CTA 0, layer l < L
 * (L = tensor-core layers) with f = 0 MMA start, 1 MMA issued, 2 epilogue
 * start, 3 epilogue done, and l = L for the input layer (f = 0 start,
 * 1 done).  Fields 4..7 of layer l < L hold SM clock cycles spent waiting
 * during that layer: the MMA issuer on activation blocks (4), on weight tiles
 * (5) and on the release of an accumulator (6); the first epilogue warp on
 * accumulators and free activation blocks (7).  On the CTA-pair shapes
 * (mode 3) fields 2..7 of l = L hold cycle sums over tile i: epilogue work
 * (2), waiting for all epilogue warps before a block is published (3),
 * pushing blocks to the peer CTA (4), and the MMA issuer's waits on
 * activation blocks produced by rank 1 (6) and by rank 0 (7).  On the
 * reverse-mode shapes (mode 4) the layer index runs over the G = 2 L' + 2
 * GEMMs of a tile (L' hidden->hidden layers: L' forward, the output layer,
 * L' backward, J_D = W_0' D_1), entry ((i * (G + 1) + g) * 8 + f) with the
 * same fields, and row g = G holds the SIMT phases: f = 0/1 the last
 * layer's adjoints, f = 2/3 the input layer of tile i.
 * rtn_tc_trace_read copies n entries to host memory (synchronous). */
#define RTN_TC_TRACE_LEN 65536
rtn_status rtn_tc_trace(rtn_ctx* ctx, int enable);
rtn_status rtn_tc_trace_read(rtn_ctx* ctx, unsigned long long* host, int n);

/* Per-launch times of the layered reverse mode (tile modes 6, 7; profiling aid).
 * enable != 0: record a CUDA event around every launch of the following
 * network passes (not inside a captured graph).  enable == 0: wait for the
 * last recorded pass, write the duration [ms] of each of its launches to
 * ms (host float [cap]) and its kind to kind (host int [cap]: 0 inputs
 * split, 1 input-layer GEMM, 2 forward GEMM, 3 output layer, 4 first
 * backward GEMM, 5 backward GEMM, 6 Jacobian GEMM), the number of launches
 * to *count, and stop recording.  Synchronous.  RTN_E_UNSUPPORTED unless the
 * context's selected tile shape is mode 6 or 7. */
rtn_status rtn_tc_launch_times(rtn_ctx* ctx, int enable, float* ms, int* kind, int cap, int* count);

/* Synchronous: the first device-side failure recorded since the last call
 * (RTN_OK if none), then clears it.  Device-side failures are bounded waits of
 * the tensor-core pipeline that gave up (RTN_E_TIMEOUT); the affected outputs
 * are then undefined. */
rtn_status rtn_device_error(rtn_ctx* ctx, int* code);

/* Budget of the bounded waits inside the layered tensor-core network kernels
 * (tile modes 6, 7; a fault-injection aid for failure-detection tests).  Every
 * mbarrier wait of those kernels gives up after `cycles` SM clock cycles
 * (0 restores the default, 4e9 cycles, about 2 s at 2 GHz): the CTA records
 * RTN_E_TIMEOUT (read and cleared by rtn_device_error), lets the copies and
 * MMAs it already issued finish (bounded by the default budget), frees its
 * tensor memory and returns; the outputs of that network pass are then
 * undefined.  A budget of a few cycles makes a pass give up at its first
 * wait that is not already satisfied.  Takes effect at the next launch;
 * RTN_E_INVAL for a negative budget. */
rtn_status rtn_set_wait_budget(rtn_ctx* ctx, long long cycles);

/* Fault injection for failure-detection tests (no GPU fault involved):
 * enable != 0 makes the TMA producer of every later layered network kernel
 * (tile modes 6, 7) first wait on a barrier that nothing completes, before it
 * issues any copy; the wait runs out after the budget of
 * rtn_set_wait_budget, the pass returns with RTN_E_TIMEOUT recorded
 * (rtn_device_error) and nothing in flight, and its outputs are undefined.
 * In the fused launch (rtn_options.fused_qp) every instance's QP waits for
 * one linearised column more than exist: each wait runs out after the same
 * budget, the instance gets status RTN_E_TIMEOUT, no step and the
 * reference input as command.  enable == 0 restores normal passes.  The
 * budget of rtn_set_wait_budget applies to the fused launch's waits too. */
rtn_status rtn_inject_wait_stall(rtn_ctx* ctx, int enable);

/* Size of the fixed activation array used by rtn_mlp_eval_f32_noalloc. */
#define RTN_NOALLOC_SCRATCH_BYTES (16u << 20)

/* FP32 network value + forward-mode Jacobian without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (and so cannot create a context with rtn_create),
 * e.g. a host that owns every device buffer itself, or a real-time loop in
 * which allocating is forbidden because it can stall the device for an
 * unbounded time.  It computes the same result as rtn_mlp_eval with
 * precision RTN_FP32, keeping the activations in a fixed array of
 * RTN_NOALLOC_SCRATCH_BYTES (16 MiB) that the library places on every GPU
 * that loads it, for the life of the process.
 *   n_layers, widths : host, as in rtn_mlp (widths[0] = 17, last = 3)
 *   W, b             : dev float, all layers packed back to back, W[l]
 *                      row-major [widths[l+1]][widths[l]], b[l] [widths[l+1]]
 *   x, u             : dev float, one row per node: x [n_nodes][13],
 *                      u [n_nodes][4]
 *   fD, JD           : dev float outputs [n_nodes][3], [n_nodes][3][17]
 *   cuda_stream      : cudaStream_t (NULL = legacy default stream)
 *   err, err_len     : optional host buffer for a message on failure
 * Requires 2 * max hidden width * 18 * n_nodes * 4 bytes <= 16 MiB, else
 * RTN_E_INVAL with the needed size in err.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current, and looks it up again when the device's context has changed
 * (after cudaDeviceReset); make that first call, and the first call after a
 * reset, before any stream capture.  All calls share
 * the one array: calls whose kernels overlap on the GPU race on it.
 * Asynchronous on cuda_stream. */
rtn_status rtn_mlp_eval_f32_noalloc(int n_layers, const int* widths, const float* W,
                                    const float* b, int n_nodes, const float* x, const float* u,
                                    float* fD, float* JD, void* cuda_stream, char* err,
                                    size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* RTN_H */
