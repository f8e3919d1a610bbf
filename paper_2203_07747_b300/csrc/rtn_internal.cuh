// rtn_internal.cuh -- context layout and kernel entry points shared by the
// CUDA translation units of librtn.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rtn.h"

// Phase tracing of the fused tensor-core network kernels (rtn_tc_trace) is a
// profiling aid compiled in only with -DRTN_TRACE=1; otherwise every trace
// branch is removed at compile time and rtn_tc_trace reports
// RTN_E_UNSUPPORTED.
#ifndef RTN_TRACE
#define RTN_TRACE 0
#endif

namespace rtn {

constexpr int NX = 13;
constexpr int NU = 4;
constexpr int NZ = 17;   // network input [x; u]
constexpr int NO = 3;    // network output: world-frame acceleration residual
constexpr int NO_FULL = 6;  // the full residual of Eq. 7: + body angular acceleration
constexpr int NC = 18;   // columns per node in forward mode: value + 17 tangents

// Quadrotor constants in FP32 for the linearisation kernels (by value).
struct QuadParams {
  float mass, inv_mass, Jx, Jy, Jz, d, c_tau, u_max, g, hover;
  // Eq. 6 torque and gyroscopic coefficients with J^-1 folded in (rounded
  // once from FP64): d / Jx, d / Jy, c_tau / Jz and (Jz - Jy) / Jx,
  // (Jx - Jz) / Jy, (Jy - Jx) / Jz
  float tq[3], gy[3];
};

// Diagonal tracking weights (Sec. V cost), kept in FP64 so that the FP64
// sweep sees the caller's exact values.
struct CostParams {
  double Q[NX], R[NU], QN[NX];
};

// Node-packed ragged layout of one controller batch.
struct Layout {
  int B = 0, n_nodes = 0, n_states = 0, N_max = 0;
  int* N = nullptr;          // [B]
  float* dt = nullptr;       // [B]
  double* dt64 = nullptr;    // [B] (plant integration)
  int* xoff = nullptr;       // [B] first state row of instance b
  int* uoff = nullptr;       // [B] first node row of instance b
  int* node_inst = nullptr;  // [n_nodes] instance of every node
  int* order = nullptr;      // [B] instances sorted by decreasing N_b
  int* rk_nodes = nullptr;   // [n_nodes] every node, instances in `order`
  int* counters = nullptr;   // [B + 3] work queue of the fused linearisation + QP launch (zero between launches)
};

// Layered reverse mode (mlp_lay.cu): values [npad][hs] and adjoints
// [3 npad][hs] as BF16 hi + lo in ping-pong buffers, d_l of every hidden
// layer [L-1][npad][hs] in FP32, tensor maps of every buffer.
struct LayState {
  int hs = 0, npad = 0;
  // activations a_1 .. a_{L-1} as BF16 hi (0) and lo (1), layer l at rows
  // (l - 1) npad; the backward epilogues recompute d_l = 1 - a_l^2 from them
  __nv_bfloat16* act[2] = {nullptr, nullptr};
  __nv_bfloat16* xb[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  alignas(64) unsigned char ma[2][128];     // activations hi / lo, box 32 x 256
  alignas(64) unsigned char mb[2][2][128];  // adjoints, box 32 x 240
  alignas(64) unsigned char mout[2][2][128];  // adjoints, box 128 x 24 unswizzled (backward GEMM's stores)
  alignas(64) unsigned char mb2[2][2][128];   // adjoints, box 32 x 120 (one CTA's half of a pair tile)
  alignas(64) unsigned char ma2[2][128];      // activations, box 32 x 128 (one CTA's half of a forward pair tile)
  bool pair_bwd = false;                      // hidden forward and backward GEMMs on CTA pairs (tile mode 7)
  alignas(64) unsigned char mact[2][128];   // activations hi / lo, box 128 x 80 unswizzled (backward epilogues)
  // folded first backward layer: M_r = W_{L-2}' diag(W_L[r]) as BF16 hi rows
  // [3 HP][HP] then lo rows, and d_{L-1} as BF16 hi + lo [npad][hs]
  __nv_bfloat16* mw = nullptr;
  __nv_bfloat16* dd[2] = {nullptr, nullptr};
  alignas(64) unsigned char mmap[128];      // M, box 32 x 128
  // input layer as a GEMM: z = [x; u] [npad][32] and W_0 [2 HP][32] (hi
  // rows, then lo rows) as BF16
  __nv_bfloat16* z[2] = {nullptr, nullptr};
  __nv_bfloat16* w0s = nullptr;
  alignas(64) unsigned char mz[2][128];     // z, box 32 x 256
  alignas(64) unsigned char mw0[128];       // W_0, box 32 x 128
  // per-launch timing of a pass (rtn_tc_launch_times): an event before
  // every launch and after the last, and each launch's kind
  // the output layer (f_D) runs on a second stream beside the first
  // backward GEMM (both read only the last forward layer's outputs)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  int n_marks = 0;
  alignas(64) unsigned char wmap[128];      // the stacked forward weights, box 32 x 128
  alignas(64) unsigned char rmap[128];      // the reverse-mode weight stack, box 32 x 128
  alignas(64) unsigned char mdd[2][128];    // d_{L-1}, box 32 x 256
  // RTN_FP8: e4m3 codes of the hidden->hidden weights W_1 .. W_{L-2} [nh HP][HP]
  // and of their transposes; activations a_1 .. a_{L-1} and adjoints as
  // three e4m3 pieces (hi, mid, lo) node-major (one byte per element)
  bool fp8 = false;
  uint8_t* q8 = nullptr;
  uint8_t* q8t = nullptr;
  uint8_t* act8[3] = {nullptr, nullptr, nullptr};
  uint8_t* xb8[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  std::vector<float> adj_scale;            // per layer l: the adjoints D_l stored as D_l * adj_scale[l]
  alignas(64) unsigned char q8map[128], q8tmap[128];  // box 64 x 128
  alignas(64) unsigned char a8map[3][128];           // box 64 x 256
  alignas(64) unsigned char b8map[2][3][128];        // box 64 x 240
  alignas(64) unsigned char a8map2[3][128];          // CTA-pair halves: box 64 x 128
  alignas(64) unsigned char b8map2[2][3][128];       // box 64 x 120
};

// Packed network for the tensor-core path -- see mlp_tc.cu.
struct TcNet {
  int h_pad = 0;                // hidden width padded to a multiple of 128
  int n_mm = 0;                 // hidden -> hidden layers on the tensor cores
  __nv_bfloat16* W = nullptr;   // stacked BF16 rows [n_mm*h_pad + 256][h_pad]
  float* bias = nullptr;        // [n_mm*h_pad + 128]
  float* W0 = nullptr;          // input layer FP32 [h_pad][17]
  float* b0 = nullptr;          // [h_pad]
  int* err = nullptr;           // device status flag (RTN_E_TIMEOUT, RTN_E_UNSUPPORTED)
  unsigned long long* trace = nullptr;  // optional phase timestamps (rtn_tc_trace)
  int rows_total = 0;
  int cols = 0, npc = 0, stages = 0, tmem_cols = 0, variant = -1, n_sm = 148;
  size_t smem = 0;
  const void* fn = nullptr;     // kernel variant
  alignas(64) unsigned char tmap_bytes[128];  // CUtensorMap of W
  // reverse mode (mlp_rev.cu): W_1..W_L, W_1'..W_{L-1}', W_0' hi, lo stacked
  __nv_bfloat16* WR = nullptr;
  float* WL32 = nullptr;                // output layer FP32 [3][h_pad]
  float* dscr = nullptr;                // per-CTA d_l scratch
  alignas(64) unsigned char tmapR_bytes[128];  // CUtensorMap of WR
  LayState* lay = nullptr;              // layered reverse mode (tile mode 6)
  long long wait_cycles = 0;            // budget of the layered kernels' bounded waits (0: default)
  int inject_stall = 0;                 // fault injection (rtn_inject_wait_stall)
};

struct Net {
  int n_layers = 0;                 // weight matrices
  std::vector<int> widths;
  float* W32 = nullptr;             // FP32 weights, all layers, row-major, packed
  float* b32 = nullptr;             // FP32 biases, packed
  std::vector<size_t> w_off, b_off; // offsets into W32 / b32
  double* P64 = nullptr;            // FP64 copy for the plant (W then b per layer)
  int h_max = 0;
  std::vector<float> fp8_scale;     // RTN_FP8: per layer, W = scale * e4m3 code
  TcNet tc;
};

// RTN_FP8: quantise n weights in place to scale * e4m3(w / scale) with
// scale = amax / 448 (round to nearest even, saturating); returns the scale
float quantize_e4m3(float* w, size_t n);

// Training buffers (allocated on the first rtn_train / rtn_mse_grad call;
// train_tc.cu).  Per layer l = 0..L-1 the input activations A_l and per
// layer output the loss gradient G_{l+1} = dLoss/dZ_{l+1}, each as BF16 hi +
// lo pairs node-major [rows][ld] (K = features) and feature-major
// [feature rows][ldf] (K = batch); the weights split hi + lo as W_l and its
// transpose; the weight gradients as one partial product per batch range.
struct TrainState {
  int cap = 0;                         // samples the buffers hold
  int rows = 0, ldf = 0;               // node rows, feature-major row length (cap rounded up to 256)
  int bs = 0;                          // samples the current plan runs on
  std::vector<__nv_bfloat16*> an, af;  // A_l node-major hi, lo (an[2l], an[2l+1]), feature-major (af)
  std::vector<__nv_bfloat16*> gn, gf;  // G_{l+1}: the same layouts
  std::vector<__nv_bfloat16*> ws;      // W_l hi, lo, W_l' hi, lo (4 per layer)
  float* z = nullptr;                  // output layer [cap][n_out]
  float* part = nullptr;               // weight-gradient partials of every layer
  std::vector<size_t> part_off;        // per layer
  std::vector<int> ksplit;             // per layer
  void* plan = nullptr;                // the step's planned GEMMs (train_tc.cu)
  float* grad = nullptr;               // dW (packed like W32) then db (like b32)
  float *m = nullptr, *v = nullptr;    // Adam moments, same packing
  size_t nw = 0, nb = 0, b_base = 0;
  long long t = 0;                     // Adam step counter (host mirror)
  int* t_dev = nullptr;                // Adam step counter on the device
  void* wjobs = nullptr;               // per-layer Adam + repack jobs of the one per-step launch
  int wjob_blocks = 0;                 // blocks of that launch
  // the weight-gradient GEMMs run on a second stream beside the backward
  // GEMMs (both read only the adjoints of the layer above): the stream and
  // one event per layer for the fork plus one for the join
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> evs;
};

// Programmatic dependent launch: the launches of a training step carry the
// programmatic-serialisation attribute, so a kernel may
// start (its prologue: barriers, tensor memory, descriptor prefetch) while
// its predecessor drains; pdl_wait() then blocks until every prerequisite
// grid has completed and its memory is visible (a no-op for an ordinary
// launch), and pdl_trigger() lets the next launch start early (once every
// CTA of this grid has called it or exited).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// a launch with the programmatic-serialisation attribute (see pdl_wait)
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

}  // namespace rtn

namespace rtn {
// Double-integrator contexts (nx = 2, nu = 1): the runtime-analysis model of
// Sec. IV, kernels in di.cu.  The residual network maps z = (p, v, u) to one
// output added to dv/dt; it is evaluated in FP32 with forward mode (value + 3
// tangents per node); the QP of each instance runs in FP32 on one thread.
struct DiState {
  int n_layers = 0;                 // 0: nominal model only
  std::vector<int> widths;          // widths[0] = 3, widths[n_layers] = 1
  std::vector<size_t> w_off, b_off;
  int h_max = 0;
  float* W = nullptr;               // every layer, row-major [out][in]
  float* b = nullptr;
  float* act0 = nullptr;            // [n_nodes][4][h_max] activations and tangents
  float* act1 = nullptr;
  double Q[2] = {0, 0}, QN[2] = {0, 0}, R = 0;
  float* lin = nullptr;             // [n_nodes][8] A, B, c of the last linearisation
  float* K = nullptr;               // [n_nodes][3] feedback gains and offsets of the last QP
};
}  // namespace rtn

namespace rtn {
// FP32-accurate network evaluation on the tensor cores (mlp_tf32.cu):
// forward mode with 18 columns per node (mode 1: value + tangents) or 176
// (mode 2: + 153 second derivatives + 5 zero pad), stored transposed,
// X' [node * columns + column][hs], as TF32 hi + lo pairs in two ping-pong
// buffers; the hidden->hidden weights split the same way, rows padded to
// kp[l] (a multiple of 32) with zeros.
struct TfState {
  int mode = 1;
  int hs = 0;                                 // row stride of X' (floats)
  float* x[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [buffer][hi, lo]
  std::vector<float*> wh, wl;                 // per hidden->hidden layer
  std::vector<int> kp;
  // per hidden->hidden layer: tensor maps of W hi, W lo, X hi, X lo
  std::vector<std::vector<unsigned char>> maps;
};
}  // namespace rtn

struct rtn_ctx {
  int B = 0;
  int nx = rtn::NX, nu = rtn::NU;   // 13, 4 (quadrotor) or 2, 1 (double integrator)
  rtn::DiState* di = nullptr;       // set for double-integrator contexts
  rtn::Layout lay;
  std::vector<int> hN;
  std::vector<double> hdt;
  rtn::QuadParams quad{};
  rtn_quad quad64{};
  rtn::CostParams cost{};
  rtn_options opt{};
  bool has_mlp = false;
  int n_out = rtn::NO;              // network outputs: 3, or 6 (full residual, rows 3-5 -> dw/dt)
  rtn::Net net;
  cudaStream_t stream = nullptr;
  // iterate (omega of Sec. II)
  float* x = nullptr;  // [n_states][13]
  float* u = nullptr;  // [n_nodes][4]
  // workspace
  float *fD = nullptr, *JD = nullptr, *A = nullptr, *Bm = nullptr, *c = nullptr;
  void *K = nullptr, *kff = nullptr;      // Riccati gains (float or double) [n][4][13], [n][4]
  // second-order local model (rtn_options.second_order): network Hessians
  // [n_nodes][n_out][17][17]; the FP32-accurate network state (mlp_tf32.cu)
  float* HD = nullptr;
  rtn::TfState* tf = nullptr;             // RTN_FP32 networks (first or second order)
  int* status = nullptr;                  // [B]
  int* dev_t = nullptr;                   // closed-loop step counter
  float* x0f = nullptr;                   // [B][13] float copy of the plant state
  float* u0 = nullptr;                    // [B][4]
  // box-constrained QP (rtn_options.box_qp): per-node scratch of the
  // active-set iterations
  float* box_dx = nullptr;                // [n_states][13] current step
  float* box_du = nullptr;                // [n_nodes][4]
  float* box_gam = nullptr;               // [n_nodes][4] diag(Huu)
  signed char* box_act = nullptr;         // [n_nodes][4] -1 lower, +1 upper, 0 free
  int* box_iters = nullptr;               // [B] subproblems of the last QP
  rtn::TrainState train;
  // rtn_rti_step_host: device copies of the step's inputs and outputs, a
  // copy stream and its events (allocated on first use)
  struct HostIO {
    cudaStream_t copy = nullptr;
    cudaEvent_t free_ev = nullptr, in_ev = nullptr;
    float *x0 = nullptr, *xref = nullptr, *uref = nullptr, *u0 = nullptr;
    int* st = nullptr;
  } hio;
  std::string err;
};

namespace rtn {

// ---- launchers (each returns cudaGetLastError()) --------------------------

// a1 / f4 for RTN_FP32 contexts (mlp_tf32.cu): f_D, J_D (and H_D in mode
// 2, second order) of every node on the tensor cores with FP32 accuracy
cudaError_t mlp_tf32_forward(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD, float* HD);
// buffers, split weights and tensor maps (at rtn_create); err receives a
// description when the tensor maps cannot be made
cudaError_t mlp_tf32_prepare(rtn_ctx* ctx, int mode, std::string& err);
void mlp_tf32_release(rtn_ctx* ctx);

// f3, double integrator (di.cu): network value + Jacobian of every node,
// linearisation (A [n][2][2], B [n][2], c [n][2]) and the RTI step
cudaError_t di_mlp(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD);
cudaError_t di_linearize(rtn_ctx* ctx, const float* x, const float* u, const float* fD,
                         const float* JD, float* A, float* Bm, float* c);
cudaError_t di_rti(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref, float* u0,
                   int* status);
cudaError_t di_reset(rtn_ctx* ctx, const float* x0);

// a1, FP32 SIMT kernels of the allocation-free entry point
cudaError_t mlp_f32_hidden_launch(const float* W, const float* bias, int M, int K, const float* X,
                                  float* Y, int n_nodes, cudaStream_t s);
cudaError_t mlp_f32_out_launch(const float* WL, const float* bL, int K, const float* X,
                               int n_nodes, float* fD, float* JD, cudaStream_t s);
// a1, tcgen05 path
cudaError_t mlp_tc_prepare(rtn_ctx* ctx, std::string& err);
cudaError_t mlp_tc_forward(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD);
void mlp_tc_release(rtn_ctx* ctx);
int mlp_tc_take_error(rtn_ctx* ctx);
int mlp_tc_variant_count();
int mlp_tc_variant_info(rtn_ctx* ctx, int idx, int* npc, int* split, int* stages);
cudaError_t mlp_tc_select(rtn_ctx* ctx, int idx);
// kernel of the CTA-pair variant (npc nodes per pair, stages weight stages), or null
// kernel of the reverse-mode variant, or null
const void* mlp_rev_fn(int npc, int stages);
// arguments of the reverse-mode kernel (mlp_rev.cu)
cudaError_t mlp_rev_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD);
// the reverse-mode kernel on CTA pairs (mlp_rev2.cu)
const void* mlp_rev2_fn(int npc, int stages);
size_t mlp_rev2_smem(int HP, int stages);
cudaError_t mlp_rev2_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD);
// layered reverse mode (mlp_lay.cu): kernel of its forward GEMM, shared
// memory of its largest GEMM, buffers and maps, launch sequence
const void* mlp_lay_fn();
size_t mlp_lay_smem();
cudaError_t mlp_lay_prepare(rtn_ctx* ctx, std::string& err);
void mlp_lay_release(rtn_ctx* ctx);
cudaError_t mlp_lay_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD);
// split-BF16 backward GEMMs of the layered path on CTA pairs (tile mode 7) or single CTAs (6)
void mlp_lay_set_pair(rtn_ctx* ctx, bool pair);
// per-launch times of the last timed pass [ms] and kinds (0 inputs, 1 input
// GEMM, 2 forward GEMM, 3 output layer, 4 first backward GEMM, 5 backward
// GEMM, 6 Jacobian GEMM); returns the number of launches
cudaError_t mlp_lay_timing(rtn_ctx* ctx, bool enable);
cudaError_t mlp_lay_times(rtn_ctx* ctx, float* ms, int* kind, int cap, int* count);

// a2
cudaError_t rk4_sens(rtn_ctx* ctx, const float* x, const float* u, const float* fD,
                     const float* JD, const float* HD, float* A, float* Bm, float* c);

// a3 + a4.  Refs are read at rows base(b) + t + k where t is *t_dev (or 0) and
// base(b) = b * stride when stride > 0, else the layout's own offset of
// instance b (node-packed references).
struct QpArgs {
  const float *A, *Bm, *c;
  float *x, *u;                 // linearisation points (updated when update != 0)
  const float *xref, *uref;
  int xref_stride, uref_stride;
  const int* t_dev;
  const float* x0;              // [B][13]
  float *dx, *du;               // optional step outputs
  float* u0;                    // optional sent command [B][4]
  int* status;                  // [B]
  int update;                   // apply step + (shift) to x, u
  int shift;
};
cudaError_t qp_solve(rtn_ctx* ctx, const QpArgs& a);
// a2 + a3 + a4 in one persistent launch (first-order 3-output model, FP32
// sweep without bounds): RK4 work units and then one QP per warp from a
// work queue; x, u, fD, JD as rk4_sens, A, Bm, c written on the way
bool lin_qp_fusable(const rtn_ctx* ctx);
cudaError_t lin_qp_solve(rtn_ctx* ctx, const QpArgs& a, const float* fD, const float* JD);

// a6 (train.cu: targets; train_tc.cu: the training step on the tensor cores)
cudaError_t drag_targets(rtn_ctx* ctx, const float* X, int n, float* Y);
// buffers for minibatches of up to cap samples, the weight splits, and the
// plan of a step on bs samples (err receives a description on failure)
cudaError_t train_prepare(rtn_ctx* ctx, TrainState& ts, int cap, int bs, std::string& err);
// loss and gradient of the minibatch [start, start + ts.bs): weight-gradient
// partials and db (into ts.grad); loss (device scalar) accumulated
cudaError_t train_grad(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                       int start, float* loss);
// the same for a step captured once and replayed: minibatch (k mod
// per_epoch) and loss entry losses[k] for k = *k_dev, which train_adam
// advances at the end of the step; its gather launch advances the Adam
// step counter ts.t_dev
cudaError_t train_grad_dev(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                           const int* k_dev, int per_epoch, float* losses);
// the partials summed into ts.grad (weights part)
cudaError_t train_reduce(rtn_ctx* ctx, TrainState& ts);
// one Adam step of every parameter from the partials and db, with the
// weight splits refreshed, in the replayed step after train_grad_dev (step
// counter ts.t_dev already advanced); then *k_dev += 1
cudaError_t train_adam(rtn_ctx* ctx, TrainState& ts, float lr, int* k_dev);
// the split weight copies of the training GEMMs from the current W32
cudaError_t train_resplit(rtn_ctx* ctx, TrainState& ts);
void train_release(rtn_ctx* ctx);

// a5
cudaError_t plant_step(rtn_ctx* ctx, int kind, const double* x, const float* u, double* xn,
                       int nsub, float* x_f32);

}  // namespace rtn
