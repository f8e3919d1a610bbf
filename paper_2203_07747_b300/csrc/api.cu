// api.cu -- the C ABI of include/rtn.h: argument checking, the node-packed
// ragged layout, device buffers and the call sequences of one RTI step
// (Sec. III-B, Fig. 2) and of a graph-captured closed loop.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "rtn_internal.cuh"

using namespace rtn;

namespace {

thread_local std::string g_create_err;

#define CK(call)                                                               \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
      return e_ == cudaErrorMemoryAllocation ? RTN_E_NOMEM : RTN_E_CUDA;       \
    }                                                                          \
  } while (0)

rtn_status fail(rtn_ctx* ctx, rtn_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

template <typename T>
cudaError_t upload(T** p, const T* h, size_t n) {
  cudaError_t e = dalloc(p, n);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*p, h, n * sizeof(T), cudaMemcpyHostToDevice);
}

__global__ void reset_kernel(const float* __restrict__ x0, const int* __restrict__ N,
                             const int* __restrict__ xoff, const int* __restrict__ uoff, int B,
                             float hover, float* __restrict__ x, float* __restrict__ u) {
  int b = blockIdx.x;
  if (b >= B) return;
  int n = N[b];
  for (int e = threadIdx.x; e < (n + 1) * NX; e += blockDim.x)
    x[(size_t)xoff[b] * NX + e] = x0[(size_t)b * NX + e % NX];
  for (int e = threadIdx.x; e < n * NU; e += blockDim.x) u[(size_t)uoff[b] * NU + e] = hover;
}

// closed loop bookkeeping: record the plant state / sent command of step t
__global__ void record_kernel(const int* t_dev, int B, const double* __restrict__ xp,
                              const float* __restrict__ u0, float* traj, float* uo) {
  int t = *t_dev;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * NX; e += gridDim.x * blockDim.x) {
    if (traj) traj[(size_t)t * B * NX + e] = (float)xp[e];
    if (uo && e < B * NU) uo[(size_t)t * B * NU + e] = u0[e];
  }
}

__global__ void advance_kernel(int* t_dev) { *t_dev += 1; }

__global__ void convert_state_kernel(const double* __restrict__ x, float* __restrict__ y, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

// f_D, J_D of every node (second-order contexts also refresh H_D)
rtn_status run_mlp(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  cudaError_t e = ctx->opt.precision == RTN_FP32 ? mlp_tf32_forward(ctx, x, u, fD, JD, ctx->HD)
                                                 : mlp_tc_forward(ctx, x, u, fD, JD);
  if (e != cudaSuccess) return fail(ctx, RTN_E_CUDA, std::string("mlp: ") + cudaGetErrorString(e));
  return RTN_OK;
}

rtn_status linearize_impl(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD,
                          float* A, float* Bm, float* c) {
  if (ctx->has_mlp) {
    rtn_status st = run_mlp(ctx, x, u, fD, JD);
    if (st != RTN_OK) return st;
  }
  cudaError_t e = rk4_sens(ctx, x, u, ctx->has_mlp ? fD : nullptr, ctx->has_mlp ? JD : nullptr,
                           ctx->opt.second_order ? ctx->HD : nullptr, A, Bm, c);
  if (e != cudaSuccess) return fail(ctx, RTN_E_CUDA, std::string("rk4: ") + cudaGetErrorString(e));
  return RTN_OK;
}

// one RTI step on the context's iterate; refs addressed by strides (0 =
// node-packed), t read from t_dev when given
// the QP, feedback and iterate update of an RTI step whose linearisation
// is in ctx->A, Bm, c
// The part of an RTI step that needs only the iterate (Sec. III-B's
// preparation): the network pass and, unless the RK4 linearisation runs in
// the fused launch with the QP, the RK4 linearisation
rtn_status rti_prep(rtn_ctx* ctx) {
  if (lin_qp_fusable(ctx)) return ctx->has_mlp ? run_mlp(ctx, ctx->x, ctx->u, ctx->fD, ctx->JD) : RTN_OK;
  return linearize_impl(ctx, ctx->x, ctx->u, ctx->fD, ctx->JD, ctx->A, ctx->Bm, ctx->c);
}

static rtn_status rti_qp(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref,
                         int xref_stride, int uref_stride, const int* t_dev, float* u0, int* status) {
  QpArgs a{};
  a.A = ctx->A; a.Bm = ctx->Bm; a.c = ctx->c;
  a.x = ctx->x; a.u = ctx->u;
  a.xref = xref; a.uref = uref;
  a.xref_stride = xref_stride; a.uref_stride = uref_stride;
  a.t_dev = t_dev;
  a.x0 = x0;
  a.u0 = u0;
  a.status = status ? status : ctx->status;
  a.update = 1;
  a.shift = ctx->opt.shift;
  cudaError_t e = lin_qp_fusable(ctx) ? lin_qp_solve(ctx, a, ctx->has_mlp ? ctx->fD : nullptr,
                                                     ctx->has_mlp ? ctx->JD : nullptr)
                                      : qp_solve(ctx, a);
  if (e != cudaSuccess) return fail(ctx, RTN_E_CUDA, std::string("qp: ") + cudaGetErrorString(e));
  return RTN_OK;
}

rtn_status rti_impl(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref,
                    int xref_stride, int uref_stride, const int* t_dev, float* u0, int* status) {
  rtn_status st = rti_prep(ctx);
  if (st != RTN_OK) return st;
  return rti_qp(ctx, x0, xref, uref, xref_stride, uref_stride, t_dev, u0, status);
}

// ragged node-packed layout of the batch (both models)
rtn_status make_layout(rtn_ctx* ctx, int batch, const int* N, const double* dt) {
  Layout& L = ctx->lay;
  L.B = batch;
  std::vector<int> xoff(batch), uoff(batch), order(batch), node_inst;
  std::vector<float> dtf(batch);
  int xs = 0, us = 0;
  for (int b = 0; b < batch; ++b) {
    xoff[b] = xs; uoff[b] = us;
    xs += N[b] + 1; us += N[b];
    dtf[b] = (float)dt[b];
    L.N_max = std::max(L.N_max, N[b]);
  }
  L.n_nodes = us; L.n_states = xs;
  node_inst.resize(us);
  for (int b = 0; b < batch; ++b)
    for (int k = 0; k < N[b]; ++k) node_inst[uoff[b] + k] = b;
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return N[a] > N[c]; });
  // every node, instances in that order (the fused linearisation + QP
  // launch hands out RK4 work in this order)
  std::vector<int> rk_nodes;
  rk_nodes.reserve(us);
  for (int b : order)
    for (int k = 0; k < N[b]; ++k) rk_nodes.push_back(uoff[b] + k);
  CK(upload(&L.rk_nodes, rk_nodes.data(), us));
  CK(dalloc(&L.counters, (size_t)batch + 3));
  CK(cudaMemset(L.counters, 0, ((size_t)batch + 3) * sizeof(int)));
  CK(upload(&L.N, N, batch));
  CK(upload(&L.dt, dtf.data(), batch));
  CK(upload(&L.dt64, dt, batch));
  CK(upload(&L.xoff, xoff.data(), batch));
  CK(upload(&L.uoff, uoff.data(), batch));
  CK(upload(&L.node_inst, node_inst.data(), us));
  CK(upload(&L.order, order.data(), batch));
  return RTN_OK;
}

// double-integrator context (nx = 2, nu = 1): the runtime-analysis model of
// Sec. IV; network z = (p, v, u) -> 1 output, FP32, no input bounds
rtn_status create_di(rtn_ctx* ctx, int batch, const int* N, const double* dt, const double* Q,
                     const double* R, const double* Q_N, const rtn_mlp* mlp, const rtn_options& o,
                     void* cuda_stream) {
  ctx->B = batch;
  ctx->nx = 2;
  ctx->nu = 1;
  ctx->opt = o;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->hN.assign(N, N + batch);
  ctx->hdt.assign(dt, dt + batch);
  ctx->di = new (std::nothrow) DiState();
  if (!ctx->di) return fail(ctx, RTN_E_NOMEM, "out of host memory");
  DiState& D = *ctx->di;
  for (int i = 0; i < 2; ++i) {
    D.Q[i] = Q[i];
    D.QN[i] = Q_N ? Q_N[i] : Q[i];
  }
  D.R = R[0];
  rtn_status st = make_layout(ctx, batch, N, dt);
  if (st != RTN_OK) return st;
  const int us = ctx->lay.n_nodes, xs = ctx->lay.n_states;
  if (mlp) {
    ctx->has_mlp = true;
    D.n_layers = mlp->n_layers;
    D.widths.assign(mlp->widths, mlp->widths + mlp->n_layers + 1);
    std::vector<float> Wh, bh;
    for (int l = 0; l < D.n_layers; ++l) {
      const int fi = D.widths[l], fo = D.widths[l + 1];
      D.w_off.push_back(Wh.size());
      D.b_off.push_back(bh.size());
      Wh.insert(Wh.end(), mlp->W[l], mlp->W[l] + (size_t)fo * fi);
      bh.insert(bh.end(), mlp->b[l], mlp->b[l] + fo);
      D.h_max = std::max(D.h_max, std::max(fi, fo));
    }
    CK(upload(&D.W, Wh.data(), Wh.size()));
    CK(upload(&D.b, bh.data(), bh.size()));
    const size_t na = (size_t)4 * D.h_max * us;
    CK(dalloc(&D.act0, na));
    CK(dalloc(&D.act1, na));
  }
  CK(dalloc(&ctx->x, (size_t)xs * 2));
  CK(dalloc(&ctx->u, (size_t)us));
  CK(dalloc(&ctx->fD, (size_t)us));
  CK(dalloc(&ctx->JD, (size_t)us * 3));
  CK(dalloc(&D.lin, (size_t)us * 8));
  CK(dalloc(&D.K, (size_t)us * 3));
  CK(dalloc(&ctx->status, batch));
  CK(dalloc(&ctx->x0f, (size_t)batch * 2));
  CK(dalloc(&ctx->u0, (size_t)batch));
  CK(cudaMemset(ctx->x0f, 0, sizeof(float) * batch * 2));
  CK(di_reset(ctx, ctx->x0f));
  CK(cudaDeviceSynchronize());
  return RTN_OK;
}

// entry points that the double-integrator model does not provide
rtn_status di_unsupported(rtn_ctx* ctx, const char* what) {
  return fail(ctx, RTN_E_UNSUPPORTED, std::string(what) + ": not available for the double-integrator model");
}

}  // namespace

extern "C" {

rtn_status rtn_create(rtn_ctx** out, int nx, int nu, int batch, const int* N, const double* dt,
                      const double* Q, const double* R, const double* Q_N, const rtn_quad* quad,
                      const rtn_mlp* mlp, const rtn_options* opt, void* cuda_stream) {
  if (!out) return RTN_E_INVAL;
  *out = nullptr;
  const bool di = nx == 2 && nu == 1;
  if (!di && (nx != NX || nu != NU)) {
    g_create_err = "nx, nu must be 13, 4 (quadrotor) or 2, 1 (double integrator)";
    return RTN_E_INVAL;
  }
  if (batch < 1 || !N || !dt || !Q || !R || (!di && !quad)) { g_create_err = "bad batch/arrays"; return RTN_E_INVAL; }
  long long nn = 0;
  for (int b = 0; b < batch; ++b) {
    if (N[b] < 1 || !(dt[b] > 0.0)) { g_create_err = "N[b] >= 1 and dt[b] > 0 required"; return RTN_E_INVAL; }
    nn += N[b];
  }
  if (nn + batch > (1LL << 28)) { g_create_err = "batch too large"; return RTN_E_INVAL; }
  rtn_options o{RTN_FP32, 0, 1, 0, 0, 0, 0, 0, 0};
  if (opt) o = *opt;
  if (o.precision < RTN_FP32 || o.precision > RTN_FP8) { g_create_err = "bad precision"; return RTN_E_INVAL; }
  if (o.box_max_iter < 0) { g_create_err = "box_max_iter must be >= 0"; return RTN_E_INVAL; }
  if (o.riccati_f64 < 0 || o.riccati_f64 > 2) { g_create_err = "riccati_f64 must be 0, 1 or 2"; return RTN_E_INVAL; }
  o.fused_qp = o.fused_qp ? 1 : 0;
  o.train_bf16 = o.train_bf16 ? 1 : 0;
  if (o.qp_group != 0 && o.qp_group != 16 && o.qp_group != 32 && o.qp_group != 256) {
    g_create_err = "qp_group must be 0, 16, 32 or 256";
    return RTN_E_INVAL;
  }
  if (o.box_max_iter == 0) o.box_max_iter = 20;
  o.box_qp = o.box_qp ? 1 : 0;
  o.second_order = o.second_order ? 1 : 0;
  if (o.second_order && (di || !mlp || o.precision != RTN_FP32)) {
    g_create_err = "second_order needs the quadrotor model, a network and RTN_FP32";
    return RTN_E_UNSUPPORTED;
  }
  if (di) {
    if (o.precision != RTN_FP32 || o.box_qp || o.riccati_f64) {
      g_create_err = "the double-integrator model runs in FP32 (network and QP), without bounds";
      return RTN_E_UNSUPPORTED;
    }
    if (mlp) {
      if (mlp->n_layers < 2 || !mlp->widths || !mlp->W || !mlp->b || mlp->widths[0] != 3 ||
          mlp->widths[mlp->n_layers] != 1) {
        g_create_err = "double-integrator network must map 3 inputs (p, v, u) to 1 output with >= 1 hidden layer";
        return RTN_E_INVAL;
      }
      for (int l = 1; l < mlp->n_layers; ++l)
        if (mlp->widths[l] < 1 || mlp->widths[l] > 65536) { g_create_err = "bad hidden width"; return RTN_E_INVAL; }
    }
    rtn_ctx* ctx = new (std::nothrow) rtn_ctx();
    if (!ctx) return RTN_E_NOMEM;
    rtn_status st = create_di(ctx, batch, N, dt, Q, R, Q_N, mlp, o, cuda_stream);
    if (st != RTN_OK) {
      g_create_err = ctx->err;
      rtn_destroy(ctx);
      return st;
    }
    *out = ctx;
    return RTN_OK;
  }
  if (mlp) {
    if (mlp->n_layers < 2 || !mlp->widths || !mlp->W || !mlp->b || mlp->widths[0] != NZ ||
        (mlp->widths[mlp->n_layers] != NO && mlp->widths[mlp->n_layers] != NO_FULL)) {
      g_create_err = "network must map 17 inputs to 3 outputs (or 6: full residual) with >= 1 hidden layer";
      return RTN_E_INVAL;
    }
    if (o.precision == RTN_FP8 && mlp->n_layers < 3) {
      g_create_err = "RTN_FP8 needs at least one hidden->hidden layer (the FP8 GEMMs)";
      return RTN_E_UNSUPPORTED;
    }
    if (mlp->widths[mlp->n_layers] == NO_FULL && o.precision != RTN_FP32) {
      g_create_err = "the 6-output full residual runs on the FP32 path (the tensor-core kernels take 3 outputs)";
      return RTN_E_UNSUPPORTED;
    }
    for (int l = 1; l < mlp->n_layers; ++l)
      if (mlp->widths[l] < 1 || mlp->widths[l] > 4096) { g_create_err = "bad hidden width"; return RTN_E_INVAL; }
  }

  rtn_ctx* ctx = new (std::nothrow) rtn_ctx();
  if (!ctx) return RTN_E_NOMEM;
  rtn_status st = RTN_OK;
  // every allocation below goes through this lambda so that a failure frees
  // what was built so far
  auto build = [&]() -> rtn_status {
    ctx->B = batch;
    ctx->opt = o;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->hN.assign(N, N + batch);
    ctx->hdt.assign(dt, dt + batch);
    ctx->quad64 = *quad;
    QuadParams& qp = ctx->quad;
    qp.mass = (float)quad->mass; qp.inv_mass = (float)(1.0 / quad->mass);
    qp.Jx = (float)quad->Jx; qp.Jy = (float)quad->Jy; qp.Jz = (float)quad->Jz;
    qp.d = (float)(quad->arm / std::sqrt(2.0)); qp.c_tau = (float)quad->c_tau;
    qp.u_max = (float)quad->u_max; qp.g = (float)quad->g;
    qp.hover = (float)(quad->mass * quad->g / 4.0);
    {
      const double d = quad->arm / std::sqrt(2.0);
      qp.tq[0] = (float)(d / quad->Jx); qp.tq[1] = (float)(d / quad->Jy); qp.tq[2] = (float)(quad->c_tau / quad->Jz);
      qp.gy[0] = (float)((quad->Jz - quad->Jy) / quad->Jx);
      qp.gy[1] = (float)((quad->Jx - quad->Jz) / quad->Jy);
      qp.gy[2] = (float)((quad->Jy - quad->Jx) / quad->Jz);
    }
    for (int i = 0; i < NX; ++i) { ctx->cost.Q[i] = Q[i]; ctx->cost.QN[i] = Q_N ? Q_N[i] : Q[i]; }
    for (int i = 0; i < NU; ++i) ctx->cost.R[i] = R[i];

    // ragged layout
    Layout& L = ctx->lay;
    rtn_status lst = make_layout(ctx, batch, N, dt);
    if (lst != RTN_OK) return lst;
    const int xs = L.n_states, us = L.n_nodes;

    // network
    if (mlp) {
      ctx->has_mlp = true;
      ctx->n_out = mlp->widths[mlp->n_layers];
      Net& net = ctx->net;
      net.n_layers = mlp->n_layers;
      net.widths.assign(mlp->widths, mlp->widths + mlp->n_layers + 1);
      std::vector<float> Wh, bh;
      std::vector<double> P64;
      for (int l = 0; l < net.n_layers; ++l) {
        int fi = net.widths[l], fo = net.widths[l + 1];
        net.w_off.push_back(Wh.size());
        net.b_off.push_back(bh.size());
        Wh.insert(Wh.end(), mlp->W[l], mlp->W[l] + (size_t)fo * fi);
        // RTN_FP8: the layer quantised to e4m3 with scale amax/448; the
        // context's network is the dequantised one (every path and the plant
        // see the same weights)
        if (o.precision == RTN_FP8) net.fp8_scale.push_back(quantize_e4m3(Wh.data() + net.w_off[l], (size_t)fo * fi));
        bh.insert(bh.end(), mlp->b[l], mlp->b[l] + fo);
        P64.insert(P64.end(), Wh.begin() + net.w_off[l], Wh.begin() + net.w_off[l] + (size_t)fo * fi);
        P64.insert(P64.end(), mlp->b[l], mlp->b[l] + fo);
        net.h_max = std::max(net.h_max, std::max(fi, fo));
      }
      CK(upload(&net.W32, Wh.data(), Wh.size()));
      CK(upload(&net.b32, bh.data(), bh.size()));
      CK(upload(&net.P64, P64.data(), P64.size()));
      if (o.precision == RTN_FP32) {
        if (o.second_order) CK(dalloc(&ctx->HD, (size_t)us * ctx->n_out * NZ * NZ));
        std::string e;
        cudaError_t ce = mlp_tf32_prepare(ctx, o.second_order ? 2 : 1, e);
        if (ce != cudaSuccess || !e.empty()) {
          ctx->err = e.empty() ? std::string("FP32 network prepare: ") + cudaGetErrorString(ce) : e;
          return ce == cudaErrorMemoryAllocation ? RTN_E_NOMEM : (e.empty() ? RTN_E_CUDA : RTN_E_UNSUPPORTED);
        }
      } else {
        std::string e;
        cudaError_t ce = mlp_tc_prepare(ctx, e);
        if (ce != cudaSuccess || !e.empty()) {
          ctx->err = e.empty() ? std::string("tc prepare: ") + cudaGetErrorString(ce) : e;
          return e.empty() ? RTN_E_CUDA : RTN_E_UNSUPPORTED;
        }
      }
    } else if (o.precision != RTN_FP32) {
      // nominal model only: nothing to run on the tensor cores
      ctx->opt.precision = RTN_FP32;
    }

    // the device status word of the fused launch's bounded waits (network
    // contexts already have one)
    if (o.fused_qp && !ctx->net.tc.err) {
      CK(dalloc(&ctx->net.tc.err, 1));
      CK(cudaMemset(ctx->net.tc.err, 0, sizeof(int)));
    }
    // iterate and workspace
    size_t gsz = ctx->opt.riccati_f64 == 1 ? sizeof(double) : sizeof(float);
    CK(dalloc(&ctx->x, (size_t)xs * NX));
    CK(dalloc(&ctx->u, (size_t)us * NU));
    CK(dalloc(&ctx->fD, (size_t)us * ctx->n_out));
    CK(dalloc(&ctx->JD, (size_t)us * ctx->n_out * NZ));
    CK(dalloc(&ctx->A, (size_t)us * NX * NX));
    CK(dalloc(&ctx->Bm, (size_t)us * NX * NU));
    CK(dalloc(&ctx->c, (size_t)us * NX));
    CK(cudaMalloc(&ctx->K, (size_t)us * NU * NX * gsz));
    CK(cudaMalloc(&ctx->kff, (size_t)us * NU * gsz));
    CK(dalloc(&ctx->status, batch));
    CK(dalloc(&ctx->dev_t, 1));
    CK(dalloc(&ctx->x0f, (size_t)batch * NX));
    CK(dalloc(&ctx->u0, (size_t)batch * NU));
    if (o.box_qp) {
      CK(dalloc(&ctx->box_dx, (size_t)xs * NX));
      CK(dalloc(&ctx->box_du, (size_t)us * NU));
      CK(dalloc(&ctx->box_gam, (size_t)us * NU));
      CK(cudaMalloc(&ctx->box_act, (size_t)us * NU));
      CK(dalloc(&ctx->box_iters, batch));
      CK(cudaMemset(ctx->box_iters, 0, sizeof(int) * batch));
    }
    // initial iterate: hover at the origin
    std::vector<float> x0(batch * NX, 0.0f);
    for (int b = 0; b < batch; ++b) x0[b * NX + 3] = 1.0f;
    CK(cudaMemcpy(ctx->x0f, x0.data(), x0.size() * sizeof(float), cudaMemcpyHostToDevice));
    reset_kernel<<<batch, 128>>>(ctx->x0f, L.N, L.xoff, L.uoff, batch, qp.hover, ctx->x, ctx->u);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    return RTN_OK;
  };
  st = build();
  if (st != RTN_OK) {
    g_create_err = ctx->err;
    rtn_destroy(ctx);
    return st;
  }
  *out = ctx;
  return RTN_OK;
}

void rtn_destroy(rtn_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  Layout& L = ctx->lay;
  void* ptrs[] = {L.N, L.dt, L.dt64, L.xoff, L.uoff, L.node_inst, L.order, L.rk_nodes, L.counters, ctx->net.W32, ctx->net.b32,
                  ctx->net.P64, ctx->x, ctx->u, ctx->fD, ctx->JD, ctx->A, ctx->Bm, ctx->c, ctx->K,
                  ctx->kff, ctx->status, ctx->dev_t, ctx->x0f, ctx->u0,
                  ctx->box_dx, ctx->box_du, ctx->box_gam, ctx->box_act, ctx->box_iters, ctx->HD};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->di) {
    void* dp[] = {ctx->di->W, ctx->di->b, ctx->di->act0, ctx->di->act1, ctx->di->lin, ctx->di->K};
    for (void* p : dp)
      if (p) cudaFree(p);
    delete ctx->di;
  }
  {
    auto& io = ctx->hio;
    void* hp[] = {io.x0, io.xref, io.uref, io.u0, io.st};
    for (void* p : hp)
      if (p) cudaFree(p);
    if (io.free_ev) cudaEventDestroy(io.free_ev);
    if (io.in_ev) cudaEventDestroy(io.in_ev);
    if (io.copy) cudaStreamDestroy(io.copy);
  }
  mlp_tf32_release(ctx);
  mlp_tc_release(ctx);
  train_release(ctx);
  delete ctx;
}

rtn_status rtn_box_iterations(rtn_ctx* ctx, int* iters) {
  if (!ctx) return RTN_E_INVAL;
  if (!iters) { ctx->err = "rtn_box_iterations: NULL output"; return RTN_E_INVAL; }
  if (!ctx->opt.box_qp) { ctx->err = "rtn_box_iterations: context has no box-constrained QP"; return RTN_E_UNSUPPORTED; }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(iters, ctx->box_iters, sizeof(int) * ctx->B, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { ctx->err = cudaGetErrorString(e); return RTN_E_CUDA; }
  return RTN_OK;
}

const char* rtn_last_error(const rtn_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

rtn_status rtn_sizes(const rtn_ctx* ctx, int* n_nodes, int* n_states) {
  if (!ctx) return RTN_E_INVAL;
  if (n_nodes) *n_nodes = ctx->lay.n_nodes;
  if (n_states) *n_states = ctx->lay.n_states;
  return RTN_OK;
}

rtn_status rtn_reset(rtn_ctx* ctx, const float* x0) {
  if (!ctx) return RTN_E_INVAL;
  if (!x0) return fail(ctx, RTN_E_INVAL, "rtn_reset: NULL argument");
  if (ctx->di) {
    CK(di_reset(ctx, x0));
    return RTN_OK;
  }
  reset_kernel<<<ctx->B, 128, 0, ctx->stream>>>(x0, ctx->lay.N, ctx->lay.xoff, ctx->lay.uoff,
                                                 ctx->B, ctx->quad.hover, ctx->x, ctx->u);
  CK(cudaGetLastError());
  return RTN_OK;
}

rtn_status rtn_set_iterate(rtn_ctx* ctx, const float* x, const float* u) {
  if (!ctx) return RTN_E_INVAL;
  if (!x || !u) return fail(ctx, RTN_E_INVAL, "rtn_set_iterate: NULL argument");
  CK(cudaMemcpyAsync(ctx->x, x, (size_t)ctx->lay.n_states * ctx->nx * sizeof(float),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->u, u, (size_t)ctx->lay.n_nodes * ctx->nu * sizeof(float),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return RTN_OK;
}

rtn_status rtn_get_iterate(rtn_ctx* ctx, float* x, float* u) {
  if (!ctx) return RTN_E_INVAL;
  if (!x || !u) return fail(ctx, RTN_E_INVAL, "rtn_get_iterate: NULL argument");
  CK(cudaMemcpyAsync(x, ctx->x, (size_t)ctx->lay.n_states * ctx->nx * sizeof(float),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(u, ctx->u, (size_t)ctx->lay.n_nodes * ctx->nu * sizeof(float),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return RTN_OK;
}

rtn_status rtn_mlp_eval(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  if (!ctx) return RTN_E_INVAL;
  if (!x || !u || !fD || !JD) return fail(ctx, RTN_E_INVAL, "rtn_mlp_eval: NULL argument");
  if (!ctx->has_mlp) return fail(ctx, RTN_E_UNSUPPORTED, "rtn_mlp_eval: no network");
  if (ctx->di) {
    CK(di_mlp(ctx, x, u, fD, JD));
    return RTN_OK;
  }
  return run_mlp(ctx, x, u, fD, JD);
}

rtn_status rtn_mlp_hess(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD, float* HD) {
  if (!ctx) return RTN_E_INVAL;
  if (!x || !u || !fD || !JD || !HD) return fail(ctx, RTN_E_INVAL, "rtn_mlp_hess: NULL argument");
  if (!ctx->opt.second_order) return fail(ctx, RTN_E_UNSUPPORTED, "rtn_mlp_hess: context has no second-order model");
  CK(mlp_tf32_forward(ctx, x, u, fD, JD, HD));
  return RTN_OK;
}

rtn_status rtn_linearize(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD,
                         float* A, float* B, float* c) {
  if (!ctx) return RTN_E_INVAL;
  if (!x || !u || !A || !B || !c) return fail(ctx, RTN_E_INVAL, "rtn_linearize: NULL argument");
  if (ctx->di) {
    float* f = fD ? fD : ctx->fD;
    float* J = JD ? JD : ctx->JD;
    if (ctx->has_mlp) CK(di_mlp(ctx, x, u, f, J));
    CK(di_linearize(ctx, x, u, ctx->has_mlp ? f : nullptr, J, A, B, c));
    return RTN_OK;
  }
  return linearize_impl(ctx, x, u, fD ? fD : ctx->fD, JD ? JD : ctx->JD, A, B, c);
}

rtn_status rtn_qp_solve(rtn_ctx* ctx, const float* A, const float* B, const float* c,
                        const float* x, const float* u, const float* xref, const float* uref,
                        const float* x0, float* dx, float* du, int* inst_status) {
  if (!ctx) return RTN_E_INVAL;
  if (!A || !B || !c || !x || !u || !xref || !uref || !x0 || !dx || !du || !inst_status)
    return fail(ctx, RTN_E_INVAL, "rtn_qp_solve: NULL argument");
  if (ctx->di) return di_unsupported(ctx, "rtn_qp_solve");
  QpArgs a{};
  a.A = A; a.Bm = B; a.c = c;
  a.x = const_cast<float*>(x); a.u = const_cast<float*>(u);
  a.xref = xref; a.uref = uref;
  a.x0 = x0; a.dx = dx; a.du = du; a.status = inst_status;
  a.update = 0;
  CK(qp_solve(ctx, a));
  return RTN_OK;
}

rtn_status rtn_rti_step(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref,
                        float* u0_out, int* inst_status) {
  if (!ctx) return RTN_E_INVAL;
  if (!x0 || !xref || !uref || !u0_out) return fail(ctx, RTN_E_INVAL, "rtn_rti_step: NULL argument");
  if (ctx->di) {
    CK(di_rti(ctx, x0, xref, uref, u0_out, inst_status));
    return RTN_OK;
  }
  return rti_impl(ctx, x0, xref, uref, 0, 0, nullptr, u0_out, inst_status);
}

rtn_status rtn_rti_step_host(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref,
                             float* u0_out, int* inst_status) {
  if (!ctx) return RTN_E_INVAL;
  if (!x0 || !xref || !uref || !u0_out) return fail(ctx, RTN_E_INVAL, "rtn_rti_step_host: NULL argument");
  if (ctx->di) return di_unsupported(ctx, "rtn_rti_step_host");
  auto& io = ctx->hio;
  const Layout& L = ctx->lay;
  const size_t bx0 = (size_t)L.B * NX * 4, bxr = (size_t)L.n_states * NX * 4, bur = (size_t)L.n_nodes * NU * 4;
  if (!io.st) {
    // set up on first use; a failure releases what was made, so that the
    // next call starts over (io.st, made last, marks a complete set-up)
    auto release = [&]() {
      void* hp[] = {io.x0, io.xref, io.uref, io.u0};
      for (void* p : hp)
        if (p) cudaFree(p);
      if (io.free_ev) cudaEventDestroy(io.free_ev);
      if (io.in_ev) cudaEventDestroy(io.in_ev);
      if (io.copy) cudaStreamDestroy(io.copy);
      io = rtn_ctx::HostIO{};
    };
    cudaError_t e = cudaStreamCreateWithFlags(&io.copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io.free_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io.in_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&io.x0, bx0);
    if (e == cudaSuccess) e = cudaMalloc(&io.xref, bxr);
    if (e == cudaSuccess) e = cudaMalloc(&io.uref, bur);
    if (e == cudaSuccess) e = cudaMalloc(&io.u0, (size_t)L.B * NU * 4);
    if (e == cudaSuccess) e = cudaMalloc(&io.st, (size_t)L.B * 4);
    if (e != cudaSuccess) {
      release();
      return fail(ctx, e == cudaErrorMemoryAllocation ? RTN_E_NOMEM : RTN_E_CUDA,
                  std::string("rtn_rti_step_host set-up: ") + cudaGetErrorString(e));
    }
  }
  // the inputs are read only by the QP: copy them on the side stream while
  // the network pass and RK4 run, once the previous step's QP has read the
  // device copies
  CK(cudaEventRecord(io.free_ev, ctx->stream));
  CK(cudaStreamWaitEvent(io.copy, io.free_ev, 0));
  CK(cudaMemcpyAsync(io.x0, x0, bx0, cudaMemcpyHostToDevice, io.copy));
  CK(cudaMemcpyAsync(io.xref, xref, bxr, cudaMemcpyHostToDevice, io.copy));
  CK(cudaMemcpyAsync(io.uref, uref, bur, cudaMemcpyHostToDevice, io.copy));
  CK(cudaEventRecord(io.in_ev, io.copy));
  rtn_status st = rti_prep(ctx);
  if (st != RTN_OK) return st;
  CK(cudaStreamWaitEvent(ctx->stream, io.in_ev, 0));
  st = rti_qp(ctx, io.x0, io.xref, io.uref, 0, 0, nullptr, io.u0, io.st);
  if (st != RTN_OK) return st;
  CK(cudaMemcpyAsync(u0_out, io.u0, (size_t)L.B * NU * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (inst_status) CK(cudaMemcpyAsync(inst_status, io.st, (size_t)L.B * 4, cudaMemcpyDeviceToHost, ctx->stream));
  return RTN_OK;
}

rtn_status rtn_plant_step(rtn_ctx* ctx, int kind, const double* x, const float* u, double* x_next,
                          int nsub) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_plant_step");
  if (!x || !u || !x_next || nsub < 1 || kind < 0 || kind > 2)
    return fail(ctx, RTN_E_INVAL, "rtn_plant_step: bad argument");
  cudaError_t e = plant_step(ctx, kind, x, u, x_next, nsub, nullptr);
  if (e == cudaErrorNotSupported)
    return fail(ctx, RTN_E_UNSUPPORTED, "plant network needs widths <= 64 and a network");
  CK(e);
  return RTN_OK;
}

rtn_status rtn_tc_variants(rtn_ctx* ctx, int* count) {
  if (!ctx || !count) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_tc_variants");
  *count = mlp_tc_variant_count();
  return RTN_OK;
}

rtn_status rtn_tc_variant_info(rtn_ctx* ctx, int idx, int* npc, int* split, int* stages,
                               int* fits) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_tc_variant_info");
  if (!ctx->has_mlp || ctx->opt.precision == RTN_FP32)
    return fail(ctx, RTN_E_UNSUPPORTED, "no tensor-core network on this context");
  int r = mlp_tc_variant_info(ctx, idx, npc, split, stages);
  if (r < 0) return fail(ctx, RTN_E_INVAL, "variant index out of range");
  if (fits) *fits = (r == 0);
  return RTN_OK;
}

rtn_status rtn_tc_select(rtn_ctx* ctx, int idx) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_tc_select");
  if (!ctx->has_mlp || ctx->opt.precision == RTN_FP32)
    return fail(ctx, RTN_E_UNSUPPORTED, "no tensor-core network on this context");
  int r = mlp_tc_variant_info(ctx, idx, nullptr, nullptr, nullptr);
  if (r < 0) return fail(ctx, RTN_E_INVAL, "variant index out of range");
  if (r > 0) return fail(ctx, RTN_E_UNSUPPORTED, "variant does not fit this network");
  CK(mlp_tc_select(ctx, idx));
  return RTN_OK;
}

rtn_status rtn_autotune(rtn_ctx* ctx, int* best_idx, float* best_ms) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_autotune");
  if (!ctx->has_mlp || ctx->opt.precision == RTN_FP32)
    return fail(ctx, RTN_E_UNSUPPORTED, "no tensor-core network on this context");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = -1;
  float bms = 1e30f;
  const int n = mlp_tc_variant_count();
  rtn_status st = RTN_OK;
  for (int i = 0; i < n && st == RTN_OK; ++i) {
    if (mlp_tc_variant_info(ctx, i, nullptr, nullptr, nullptr) != 0) continue;
    cudaError_t e = mlp_tc_select(ctx, i);
    if (e == cudaSuccess) e = mlp_tc_forward(ctx, ctx->x, ctx->u, ctx->fD, ctx->JD);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = mlp_tc_forward(ctx, ctx->x, ctx->u, ctx->fD, ctx->JD);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { ctx->err = std::string("autotune: ") + cudaGetErrorString(e); st = RTN_E_CUDA; break; }
    if (mlp_tc_take_error(ctx)) { ctx->err = "autotune: device timeout"; st = RTN_E_TIMEOUT; break; }
    ms /= 3.0f;
    if (ms < bms) { bms = ms; best = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RTN_OK) return st;
  if (best < 0) return fail(ctx, RTN_E_UNSUPPORTED, "no variant fits");
  CK(mlp_tc_select(ctx, best));
  if (best_idx) *best_idx = best;
  if (best_ms) *best_ms = bms;
  return RTN_OK;
}

rtn_status rtn_tc_trace(rtn_ctx* ctx, int enable) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_tc_trace");
  TcNet& tc = ctx->net.tc;
  if (!ctx->has_mlp || ctx->opt.precision == RTN_FP32)
    return fail(ctx, RTN_E_UNSUPPORTED, "no tensor-core network on this context");
  if (!RTN_TRACE && enable)
    return fail(ctx, RTN_E_UNSUPPORTED, "rtn_tc_trace: built without phase tracing (compile with -DRTN_TRACE=1)");
  if (enable && !tc.trace) {
    CK(cudaMalloc(&tc.trace, RTN_TC_TRACE_LEN * sizeof(unsigned long long)));
    CK(cudaMemset(tc.trace, 0, RTN_TC_TRACE_LEN * sizeof(unsigned long long)));
  } else if (!enable && tc.trace) {
    CK(cudaFree(tc.trace));
    tc.trace = nullptr;
  }
  return RTN_OK;
}

rtn_status rtn_tc_trace_read(rtn_ctx* ctx, unsigned long long* host, int n) {
  if (!ctx || !host || n < 0 || n > RTN_TC_TRACE_LEN) return fail(ctx, RTN_E_INVAL, "rtn_tc_trace_read: bad argument");
  if (ctx->di) return di_unsupported(ctx, "rtn_tc_trace_read");
  if (!ctx->net.tc.trace) return fail(ctx, RTN_E_INVAL, "tracing is not enabled");
  CK(cudaMemcpy(host, ctx->net.tc.trace, (size_t)n * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  return RTN_OK;
}

rtn_status rtn_tc_launch_times(rtn_ctx* ctx, int enable, float* ms, int* kind, int cap, int* count) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_tc_launch_times");
  if (!ctx->net.tc.lay || ctx->net.tc.variant < 0 || mlp_tc_variant_info(ctx, ctx->net.tc.variant, nullptr, nullptr, nullptr) != 0)
    return fail(ctx, RTN_E_UNSUPPORTED, "rtn_tc_launch_times: the layered reverse mode is not selected");
  {
    int mode = 0;
    mlp_tc_variant_info(ctx, ctx->net.tc.variant, nullptr, &mode, nullptr);
    if (mode != 6 && mode != 7)
      return fail(ctx, RTN_E_UNSUPPORTED, "rtn_tc_launch_times: the layered reverse mode is not selected");
  }
  if (enable) {
    CK(mlp_lay_timing(ctx, true));
    if (count) *count = 0;
    return RTN_OK;
  }
  if (!ms || !kind || !count || cap < 0) return fail(ctx, RTN_E_INVAL, "rtn_tc_launch_times: NULL argument");
  if (!ctx->net.tc.lay->timing) return fail(ctx, RTN_E_INVAL, "rtn_tc_launch_times: timing is not enabled");
  CK(mlp_lay_times(ctx, ms, kind, cap, count));
  CK(mlp_lay_timing(ctx, false));
  return RTN_OK;
}

rtn_status rtn_device_error(rtn_ctx* ctx, int* code) {
  if (!ctx || !code) return RTN_E_INVAL;
  if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
  else CK(cudaDeviceSynchronize());
  *code = mlp_tc_take_error(ctx);
  return RTN_OK;
}

rtn_status rtn_set_wait_budget(rtn_ctx* ctx, long long cycles) {
  if (!ctx) return RTN_E_INVAL;
  if (cycles < 0) return fail(ctx, RTN_E_INVAL, "rtn_set_wait_budget: negative budget");
  ctx->net.tc.wait_cycles = cycles;
  return RTN_OK;
}

rtn_status rtn_inject_wait_stall(rtn_ctx* ctx, int enable) {
  if (!ctx) return RTN_E_INVAL;
  ctx->net.tc.inject_stall = enable ? 1 : 0;
  return RTN_OK;
}

rtn_status rtn_closed_loop(rtn_ctx* ctx, int steps, int plant_kind, const float* xref_traj,
                           const float* uref_traj, int T, double* x_plant, float* traj_out,
                           float* u_out) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) return di_unsupported(ctx, "rtn_closed_loop");
  if (steps < 0 || !xref_traj || !uref_traj || !x_plant || plant_kind < 0 || plant_kind > 2 ||
      T < steps + ctx->lay.N_max + 1)
    return fail(ctx, RTN_E_INVAL, "rtn_closed_loop: bad argument");
  if (steps == 0) return RTN_OK;
  if (plant_kind == RTN_PLANT_MLP && (!ctx->has_mlp || ctx->net.h_max > 64))
    return fail(ctx, RTN_E_UNSUPPORTED, "plant network needs widths <= 64 and a network");
  // one control step is an RTI step (linearise at the iterate, QP from the
  // measured state) and a plant step.  Step k + 1's linearisation reads only
  // the iterate that step k's QP left, not the plant state, so the replayed
  // graph runs step k's plant step (and its record and the step counter) on
  // a second branch beside step k + 1's linearisation and joins them before
  // step k + 1's QP; the first step's RTI step and the last step's plant step
  // run outside the graph.  The kernels read the step index from
  // ctx->dev_t, which the plant branch advances.
  cudaStream_t user = ctx->stream, cs = nullptr, cs2 = nullptr;
  cudaEvent_t ev = nullptr, fork = nullptr, join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  rtn_status st = RTN_OK;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev) cudaEventDestroy(ev);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (cs) cudaStreamDestroy(cs);
    if (cs2) cudaStreamDestroy(cs2);
    ctx->stream = user;
  };
  // plant step of the current step index, its record, then the next index
  auto plant_branch = [&](cudaStream_t s) -> cudaError_t {
    ctx->stream = s;
    cudaError_t r = plant_step(ctx, plant_kind, x_plant, ctx->u0, x_plant, 4, ctx->x0f);
    record_kernel<<<(ctx->B * NX + 255) / 256, 256, 0, s>>>(ctx->dev_t, ctx->B, x_plant, ctx->u0, traj_out,
                                                            u_out);
    advance_kernel<<<1, 1, 0, s>>>(ctx->dev_t);
    ctx->stream = cs;
    return r != cudaSuccess ? r : cudaGetLastError();
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_t, 0, sizeof(int), user);
  if (e == cudaSuccess) e = cudaEventRecord(ev, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
  if (e != cudaSuccess) { ctx->err = cudaGetErrorString(e); cleanup(); return RTN_E_CUDA; }
  ctx->stream = cs;
  if (steps > 1) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = cudaEventRecord(fork, cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs2, fork, 0);
      if (e == cudaSuccess) e = plant_branch(cs2);  // step k
      if (e == cudaSuccess) {
        st = rti_prep(ctx);  // step k + 1
        ctx->stream = cs;
      }
      if (e == cudaSuccess) e = cudaEventRecord(join, cs2);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join, 0);
      // the plant state in float is the measured x0 of the RTI step
      if (e == cudaSuccess && st == RTN_OK)
        st = rti_qp(ctx, ctx->x0f, xref_traj, uref_traj, T, T - 1, ctx->dev_t, ctx->u0, ctx->status);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e2;
    }
    if (st != RTN_OK || e != cudaSuccess) {
      if (st == RTN_OK) { ctx->err = std::string("capture: ") + cudaGetErrorString(e); st = RTN_E_CUDA; }
      cleanup();
      return st;
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
  }
  if (e == cudaSuccess) {
    convert_state_kernel<<<(ctx->B * NX + 255) / 256, 256, 0, cs>>>(x_plant, ctx->x0f, ctx->B * NX);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    st = rti_impl(ctx, ctx->x0f, xref_traj, uref_traj, T, T - 1, ctx->dev_t, ctx->u0, ctx->status);
    ctx->stream = cs;
  }
  for (int s = 1; s < steps && e == cudaSuccess && st == RTN_OK; ++s) e = cudaGraphLaunch(exec, cs);
  if (e == cudaSuccess && st == RTN_OK) e = plant_branch(cs);
  if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) { ctx->err = std::string("closed loop: ") + cudaGetErrorString(e); st = RTN_E_CUDA; }
  cleanup();
  return st;
}

}  // extern "C"
